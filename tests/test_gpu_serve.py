"""Serving with continuous batching: render and gradient requests of
different meshes, resolutions and depths, arriving while others run, give
the same result as each request alone (within the tolerance of float
atomics) and, for a sample of them, the FP64 oracle's; the loop reports
latency and throughput."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, PROBE, assert_radiance_parity
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


# requests of the oracle comparison: (scene, side, depth, kind) and the
# fraction of their pixels the oracle's criterion excludes (measured with
# the oracle alone on the same seeded views)
ORACLE_CASES = [(0, 24, 13, "render", 0.0312), (1, 20, 12, "grad", 0.14), (2, 22, 6, "render", 0.1715),
                (0, 18, 5, "grad", 0.0185)]


def _np(t):
    return t.detach().cpu().numpy()


def _oracle_requests(resident):
    """The four checked requests among eight others of the same stream; the
    checked gradient requests get a target equal to their alone-run image on
    the pixels the oracle excludes, so those pixels seed no gradient."""
    rng = np.random.default_rng(61)
    trg = np.random.default_rng(62)
    filler = serve.poisson_requests(rng, 8, 1e6, 3, sides=(16, 48), depths=(3, 13), grad_frac=0.5, view_fn=_view,
                                    target_fn=lambda r: trg.uniform(0, 2, size=(r.height, r.width, 3)).astype(
                                        np.float32))
    checked = []
    for j, (scene, side, depth, kind, excl) in enumerate(ORACLE_CASES):
        cam = S.random_view(np.random.default_rng(70 + j), 3.0, side, side)
        r = serve.Request(rid=100 + j, scene=scene, cam=cam.as_array(), width=side, height=side, depth=depth,
                          kind=kind, arrival=0.0)
        sc = resident[scene]
        orc = O.render(_np(sc.V), _np(sc.F), float(_np(sc.ior)[0]), _np(sc.sigma), _np(sc.env), cam, depth,
                       probe=PROBE)
        bad = (orc["pix_flags"] & O.SEG_DEGENERATE) != 0
        if kind == "grad":
            t = trg.uniform(0, 2, size=(side, side, 3)).astype(np.float32)
            probe = serve.Request(rid=-1, scene=scene, cam=r.cam, width=side, height=side, depth=depth,
                                  kind="render", arrival=0.0)
            alone, _ = _alone(sc, probe)
            t[bad] = alone[bad]
            r.target = t
        checked.append((r, cam, orc, bad, excl))
    reqs = filler[:4] + [c[0] for c in checked] + filler[4:]
    for i, r in enumerate(reqs):
        r.arrival = 1e-4 * i
    return reqs, checked


def test_served_results_match_the_oracle(resident):
    """Served render and gradient requests (one of depth 13, one of depth 12)
    in a burst with eight others, checked against the FP64 oracle: the
    image within the radiance tolerance on the pixels its criterion keeps,
    and dLoss/dIoR, dLoss/dsigma and two random directional derivatives in
    the vertices within the gradient tolerance of the oracle's forward-mode
    derivative of the same L2 loss."""
    reqs, checked = _oracle_requests(resident)
    srv = serve.Server(resident, memory_budget=2 << 30, max_batch=8, streams=2)
    done = {r.rid: r for r in srv.run(reqs, timeout=120)}
    assert len(done) == len(reqs) and srv.launches < len(reqs)
    for r0, cam, orc, bad, excl in checked:
        r = done[r0.rid]
        sc = resident[r.scene]
        assert_radiance_parity(torch.from_numpy(r.image), orc, excl)
        if r.kind != "grad":
            continue
        # the loss the server seeds its backward with: mean (I - T)^2; its
        # gradient from the oracle's image, zero on the excluded pixels
        n = r.image.size
        g = 2.0 * (orc["img"] - r.target.astype(np.float64)) / n
        g[bad] = 0.0
        V, F = _np(sc.V), _np(sc.F)
        urng = np.random.default_rng(r.rid)
        U = urng.normal(size=(2,) + V.shape)
        tV = np.concatenate([np.zeros((4,) + V.shape), U])
        tior = np.array([1.0, 0, 0, 0, 0, 0])
        tsig = np.zeros((6, 3))
        tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
        _, dimg = O.render_jvp(V, F, float(_np(sc.ior)[0]), _np(sc.sigma), _np(sc.env), cam, r.depth, tV, tior, tsig)
        J = np.einsum("khwc,hwc->k", dimg, g)
        assert r.grad_ior == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1e-3, abs(J[0])))
        np.testing.assert_allclose(r.grad_sigma, J[1:4], rtol=GRAD_RTOL, atol=1e-6 * max(1e-3, np.abs(J[1:4]).max()))
        dV = r.grad_V.astype(np.float64)
        for j in range(2):
            proj = float((dV * U[j]).sum())
            assert abs(proj - J[4 + j]) <= GRAD_RTOL * abs(J[4 + j]) + 3 * GRAD_RTOL * np.linalg.norm(dV), (proj, J[4 + j])
