"""Serving with continuous batching: render and gradient requests of
different meshes, resolutions and depths, arriving while others run, give
the same result as each request alone (within the tolerance of float
atomics), and the loop reports latency and throughput."""
import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL
from paper_2603_00413_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def resident():
    from paper_2603_00413_gb300 import build
    build.build()
    rng = np.random.default_rng(31)
    dev = torch.device("cuda:0")
    out = []
    V, F = S.icosphere(3)
    out.append(serve.ResidentScene.from_arrays(V, F, 1.5, [0.2, 0.4, 0.6], S.sh_env_map(64, 32, 1), dev))
    V, F = S.two_tori_mesh(32)
    out.append(serve.ResidentScene.from_arrays(V, F, 1.45, [1.0, 0.5, 0.1], S.sh_env_map(64, 32, 2), dev))
    V, F = S.mesh_from_field(S.random_blob_field(rng), 4000)
    out.append(serve.ResidentScene.from_arrays(V, F, 1.6, [0.0, 0.0, 0.0], S.sh_env_map(32, 16, 3), dev))
    return out


def _view(rng, side):
    return S.random_view(rng, 3.0, side, side).as_array()


def _requests(n, rate, seed):
    rng = np.random.default_rng(seed)
    trg = np.random.default_rng(seed + 1)
    return serve.poisson_requests(rng, n, rate, 3, sides=(16, 96), depths=(2, 9), grad_frac=0.5, view_fn=_view,
                                  target_fn=lambda r: trg.uniform(0, 2, size=(r.height, r.width, 3)).astype(np.float32))


def _alone(scene, r):
    dev = scene.V.device
    cams = torch.from_numpy(r.cam.reshape(1, 10)).to(dev)
    img, tape = dt.render(scene.V, scene.F, scene.bvh, scene.N, scene.ior, scene.sigma, scene.env, cams, r.width,
                          r.height, dt.Params(r.depth))
    if r.kind == "render":
        return img[0].cpu().numpy(), None
    tgt = torch.from_numpy(r.target.reshape(1, r.height, r.width, 3)).to(dev)
    g, loss = dt.l2_loss_grad(img, tgt)
    dV, dior, dsig = dt.render_backward(tape, g)
    return img[0].cpu().numpy(), (dV.cpu().numpy(), float(dior), dsig.cpu().numpy(), float(loss))


@pytest.mark.parametrize("max_batch,streams,rate", [(8, 2, 400.0), (8, 2, 1e6), (1, 1, 400.0)])
def test_served_results_equal_alone(resident, max_batch, streams, rate):
    reqs = _requests(24, rate, 40)
    srv = serve.Server(resident, memory_budget=2 << 30, max_batch=max_batch, streams=streams)
    done = srv.run(reqs, timeout=120)
    assert len(done) == len(reqs)
    assert all(r.finish >= r.start >= r.arrival for r in done)
    if rate > 1e5:
        assert srv.launches < len(reqs)  # a burst is served in batches
    for r in sorted(done, key=lambda r: r.rid):
        img, gr = _alone(resident[r.scene], r)
        np.testing.assert_allclose(r.image, img, rtol=1e-5, atol=1e-7)
        if r.kind == "grad":
            dV, dior, dsig, loss = gr
            assert np.linalg.norm(r.grad_V - dV) <= GRAD_RTOL * max(np.linalg.norm(dV), 1e-12)
            assert r.grad_ior == pytest.approx(dior, rel=GRAD_RTOL, abs=1e-9)
            np.testing.assert_allclose(r.grad_sigma, dsig, rtol=GRAD_RTOL, atol=1e-9)
            assert r.loss == pytest.approx(loss, rel=1e-5)
    s = serve.latency_summary(done, max(r.finish for r in done))
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["segments_per_s"] > 0


def test_admission_respects_the_memory_budget(resident):
    """With a budget that fits about one request at a time the server still
    serves everything (a too-large head request runs alone)."""
    reqs = _requests(6, 2000.0, 50)
    srv = serve.Server(resident, memory_budget=1, max_batch=8, streams=2)
    done = srv.run(reqs, timeout=120)
    assert len(done) == 6
    assert srv.launches >= 6
