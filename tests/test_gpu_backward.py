"""GPU adjoint vs the FP64 oracle: gradients of J = sum(g * image) with
respect to vertex positions, IoR and per-channel absorption must agree within
1e-3 relative with the oracle's forward-mode derivative (dual numbers) and
with central finite differences of the oracle on pixels whose event signature
is the same at +h and -h."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, GpuScene, excluded_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _gpu_grads(gs, g):
    img, tape = gs.render()
    dV, dior, dsig = dt.render_backward(tape, torch.from_numpy(g.astype(np.float32)).cuda())
    return img, dV.cpu().numpy().astype(np.float64), float(dior.item()), dsig.cpu().numpy().astype(np.float64)


def _oracle_jvp(gs, view, tV=None, tior=None, tsig=None):
    p = gs.params
    return O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[view], p.max_depth, tV, tior, tsig,
                        p.spp, p.jitter, p.seed, view, p.t_min)[1]


def _masked_seed(gs, rng, expected_excluded):
    """Random image gradient, zero on the edge-degenerate pixels (whose FP32
    and FP64 paths may differ); their fraction is checked against the
    measured one."""
    orc = gs.oracle(0)
    g = rng.normal(size=(1, gs.height, gs.width, 3))
    g[0][excluded_pixels(orc, expected_excluded)] = 0.0
    return g


def _check_against_jvp(gs, rng, expected_excluded, n_dirs=4, full=False):
    g = _masked_seed(gs, rng, expected_excluded)
    _, dV, dior, dsig = _gpu_grads(gs, g)
    # exact partials for ior and sigma
    tior = np.array([1.0, 0, 0, 0])
    tsig = np.zeros((4, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    d = _oracle_jvp(gs, 0, None, tior, tsig)
    J = np.einsum("khwc,hwc->k", d, g[0])
    assert dior == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1.0, abs(J[0])))
    np.testing.assert_allclose(dsig, J[1:], rtol=GRAD_RTOL, atol=1e-6 * max(1.0, np.abs(J[1:]).max()))
    # random directional derivatives for the vertices: for u ~ N(0, I) the
    # projection of an error vector e has size ~|e|, so it is bounded
    # against the gradient's norm (3 sigma) as well as relatively
    U = rng.normal(size=(n_dirs,) + gs.Vn.shape)
    d = _oracle_jvp(gs, 0, U)
    Ju = np.einsum("khwc,hwc->k", d, g[0])
    gu = np.einsum("kvc,vc->k", U, dV)
    np.testing.assert_allclose(gu, Ju, rtol=GRAD_RTOL, atol=3 * GRAD_RTOL * np.linalg.norm(dV))
    if full:
        p = gs.params
        dVo, dioro, dsigo = O.grad_full(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth,
                                        g[0], spp=p.spp, jitter=p.jitter, seed=p.seed, t_min=p.t_min)
        rel = np.linalg.norm(dV - dVo) / np.linalg.norm(dVo)
        assert rel < GRAD_RTOL, rel
    return g, dV, dior, dsig


def test_gradients_icosphere_absorbing_match_oracle():
    sc = S.glass_icosphere_scene(width=24, height=24)
    cam = S.camera((0.4, 0.7, 2.8), (0, 0, 0), (0, 1, 0), 45.0, 24, 24)
    gs = GpuScene(sc.V, sc.F, 1.45, np.array([0.5, 1.0, 1.5], np.float32), sc.env, [cam], 24, 24, 4)
    _check_against_jvp(gs, np.random.default_rng(0), 0.0295, full=True)


def test_gradients_genus2_depth8_match_oracle():
    V, F = S.two_tori_mesh(32)
    env = S.sh_env_map(64, 32, 1)
    cam = S.fibonacci_views(5, 3.0, 24, 24)[1]
    gs = GpuScene(V, F, 1.4, np.array([1.2, 0.4, 1.9], np.float32), env, [cam], 24, 24, 8)
    _check_against_jvp(gs, np.random.default_rng(1), 0.151)


def test_gradients_match_central_differences():
    """GPU reverse mode vs central differences of the FP64 oracle, with the
    seed g restricted to pixels whose event signature is stable at +-h."""
    sc = S.glass_icosphere_scene(width=20, height=20)
    cam = S.camera((0.2, 0.3, 2.9), (0, 0, 0), (0, 1, 0), 45.0, 20, 20)
    sigma = np.array([0.7, 0.2, 1.1], np.float32)
    gs = GpuScene(sc.V, sc.F, 1.5, sigma, sc.env, [cam], 20, 20, 5)
    rng = np.random.default_rng(3)
    g0 = _masked_seed(gs, rng, 0.04)
    h = 1e-6
    p = gs.params
    V64 = gs.Vn.astype(np.float64)
    u = rng.normal(size=V64.shape)
    cases = {
        "V": (dict(V=V64 + h * u), dict(V=V64 - h * u)),
        "ior": (dict(ior=gs.iorf + h), dict(ior=gs.iorf - h)),
        "sigma0": (dict(sigma=sigma + np.array([h, 0, 0])), dict(sigma=sigma - np.array([h, 0, 0]))),
    }
    for name, (plus, minus) in cases.items():
        def run(over):
            a = dict(V=V64, ior=gs.iorf, sigma=sigma.astype(np.float64))
            a.update(over)
            return O.render(a["V"], gs.Fn, a["ior"], a["sigma"], gs.envn, cam, p.max_depth)
        rp, rm = run(plus), run(minus)
        stable = rp["pix_sig"] == rm["pix_sig"]
        g = g0 * stable[None, ..., None]
        fd = ((rp["img"] - rm["img"]) / (2 * h) * g[0]).sum()
        _, dV, dior, dsig = _gpu_grads(gs, g)
        got = {"V": (dV * u).sum(), "ior": dior, "sigma0": dsig[0]}[name]
        assert got == pytest.approx(fd, rel=GRAD_RTOL, abs=1e-7), name


def test_ior_one_gives_zero_vertex_gradient():
    sc = S.glass_icosphere_scene(width=24, height=24)
    gs = GpuScene(sc.V, sc.F, 1.0, np.zeros(3, np.float32), sc.env, sc.cams, 24, 24, 4)
    g = np.random.default_rng(4).normal(size=(1, 24, 24, 3))
    img, dV, dior, dsig = _gpu_grads(gs, g)
    assert np.abs(dV).max() < 1e-4 * max(1.0, abs(dior))


def test_autograd_function_matches_render_backward():
    sc = S.glass_icosphere_scene(width=16, height=16)
    gs = GpuScene(sc.V, sc.F, 1.45, np.array([0.5, 1.0, 1.5], np.float32), sc.env, sc.cams, 16, 16, 4)
    V = gs.V.clone().requires_grad_(True)
    ior = gs.ior.clone().requires_grad_(True)
    sigma = gs.sigma.clone().requires_grad_(True)
    target = torch.rand(1, 16, 16, 3, device="cuda")
    img = dt.render_differentiable(V, gs.F, ior, sigma, gs.env, gs.cams, 16, 16, gs.params)
    loss = ((img - target) ** 2).mean()
    loss.backward()
    g = (2.0 * (img.detach() - target) / img.numel()).cpu().numpy()
    _, dV, dior, dsig = _gpu_grads(gs, g)
    # two GPU runs: float atomics add in a different order, so entries that
    # cancel to ~0 differ at the level of rounding of the large terms
    np.testing.assert_allclose(V.grad.cpu().numpy(), dV, rtol=1e-4, atol=1e-5 * np.abs(dV).max())
    assert ior.grad.item() == pytest.approx(dior, rel=1e-4, abs=1e-9)
    np.testing.assert_allclose(sigma.grad.cpu().numpy(), dsig, rtol=1e-4, atol=1e-9)
