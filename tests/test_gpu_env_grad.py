"""Gradient with respect to the environment texels (the bilinear lookup of
Sec. 3.4 step 3, differentiated in its texels).  The
image is linear in the texels (pinned on the oracle), so the oracle's render
with the environment replaced by a direction u is the image's derivative
along u; the device's dJ/dE, projected on u, must match it.  Checked with
the shared-memory path (an environment of at most 4096 texels), the global
path (larger ones), per texel on a few texels, in a batch, and without
changing the other gradients."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, PROBE, GpuScene, excluded_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def _scene(env_w, env_h, w=28, h=24, depth=5):
    V, F = S.two_tori_mesh(36)
    return GpuScene(V, F, 1.5, np.array([0.3, 0.1, 0.05], np.float32), S.sh_env_map(env_w, env_h, 2),
                    S.fibonacci_views(1, 3.0, w, h), w, h, depth)


def _oracle_img(gs, env):
    p = gs.params
    return O.render(gs.Vn, gs.Fn, gs.iorf, gs.sigman, env, gs.cam_list[0], p.max_depth, p.spp, p.jitter, p.seed, 0,
                    p.t_min)["img"]


def _check(gs, rng, expected_excluded, n_dirs=3):
    p = gs.params
    orc = O.render(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, p.spp, p.jitter, p.seed,
                   0, p.t_min, probe=PROBE)
    g = rng.normal(size=(1, gs.height, gs.width, 3))
    g[0][excluded_pixels(orc, expected_excluded)] = 0.0
    img, tape = gs.render()
    out = dt.render_backward(tape, torch.from_numpy(g.astype(np.float32)).cuda(), env_grad=True)
    denv = out[3].cpu().numpy().astype(np.float64)
    assert denv.shape == gs.envn.shape and np.abs(denv).max() > 0
    for _ in range(n_dirs):
        u = rng.normal(size=gs.envn.shape)
        J = float((g[0] * _oracle_img(gs, u)).sum())
        proj = float((denv * u).sum())
        assert abs(proj - J) <= GRAD_RTOL * abs(J) + 3 * GRAD_RTOL * np.linalg.norm(denv), (proj, J)
    return g, out, denv


def test_env_gradient_shared_memory_path():
    _check(_scene(64, 32), np.random.default_rng(51), 0.0432)


def test_env_gradient_global_path():
    _check(_scene(128, 64), np.random.default_rng(52), 0.0432)


def test_env_gradient_per_texel():
    """Exact entries: the texels the most escaped throughput reads."""
    gs = _scene(16, 8, w=20, h=16)
    rng = np.random.default_rng(53)
    g, _, denv = _check(gs, rng, 0.0656, n_dirs=1)
    flat = np.argsort(-np.abs(denv).reshape(-1))[:4]
    for j in flat:
        e = np.zeros(denv.size)
        e[j] = 1.0
        J = float((g[0] * _oracle_img(gs, e.reshape(denv.shape))).sum())
        assert denv.reshape(-1)[j] == pytest.approx(J, rel=GRAD_RTOL, abs=1e-7)


def test_env_gradient_leaves_other_gradients_and_batches():
    gs = _scene(64, 32)
    rng = np.random.default_rng(54)
    g = torch.from_numpy(rng.normal(size=(1, gs.height, gs.width, 3)).astype(np.float32)).cuda()
    _, tape = gs.render()
    a = dt.render_backward(tape, g)
    b = dt.render_backward(tape, g, env_grad=True)
    assert len(a) == 3 and len(b) == 4
    for x, y in zip(a, b[:3]):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-5 * max(np.linalg.norm(x), 1e-12)
    sc = S.glass_icosphere_scene(width=20, height=20)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 20, 20, 4)
    g1 = torch.from_numpy(rng.normal(size=(1, 20, 20, 3)).astype(np.float32)).cuda()
    items = [dt.BatchItem(x.V, x.F, x.bvh, x.N, x.ior, x.sigma, x.env, x.cams, x.width, x.height, x.params)
             for x in (gs, ico)]
    _, bt = dt.render_batch(items)
    out = dt.render_batch_backward(bt, [g, g1], env_grad=True)
    _, t1 = ico.render()
    ref1 = dt.render_backward(t1, g1, env_grad=True)[3].cpu().numpy().astype(np.float64)
    for got, ref in ((out[0][3], b[3]), (out[1][3], ref1)):
        got = got.cpu().numpy().astype(np.float64)
        ref = ref if isinstance(ref, np.ndarray) else ref.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-4 * max(np.linalg.norm(ref), 1e-12)
