"""Spatially varying absorption (Eq. 11 with mu_t(x) = sigma + G(x), G a
dense grid of per-channel rates, trilinear, clamped to its box; interior
segments add the sum of G over steps of length h from their start, the last
one partial, sampled at midpoints).  The CUDA forward and adjoint against
the FP64 oracle: radiance, the gradient with respect to the node values
(along random directions, against the oracle's forward-mode derivative),
IoR and sigma; the vertex gradient where G is linear (so its gradient has no
jumps at cell faces); a constant grid against a sigma shift; the grid in a
batch next to a scene without one; and the checkpointed tape."""
import copy

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, PROBE, GpuScene, assert_radiance_parity, excluded_pixels

pytestmark = pytest.mark.gpu

LO, HI = (-1.25, -1.25, -1.25), (1.25, 1.25, 1.25)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def _gpu_medium(med):
    mu = torch.from_numpy(np.asarray(med["mu"], np.float32)).cuda()
    return dt.Medium(mu, med["lo"], med["hi"], med["step"])


def _oracle_medium(med):
    """The same grid as the device sees it: float32 node values, box and
    step (as doubles)."""
    return dict(mu=np.asarray(med["mu"], np.float32).astype(np.float64),
                lo=tuple(float(np.float32(x)) for x in med["lo"]),
                hi=tuple(float(np.float32(x)) for x in med["hi"]), step=float(np.float32(med["step"])))


def _scene(w=40, h=32, views=2, depth=6, sigma=(0.2, 0.05, 0.1), mesh="tori"):
    if mesh == "tori":
        V, F = S.two_tori_mesh(36)
    else:
        V, F = S.icosphere(3, 1.0)
    return GpuScene(V, F, 1.5, np.array(sigma, np.float32), S.sh_env_map(64, 32, 1),
                    S.fibonacci_views(views, 3.0, w, h), w, h, depth, spp=1, jitter=0, seed=0)


def _oracle(gs, med, view=0, probe=PROBE):
    p = gs.params
    return O.render(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[view], p.max_depth, p.spp, p.jitter,
                    p.seed, view, p.t_min, probe=probe, medium=_oracle_medium(med))


def test_medium_render_matches_oracle():
    gs = _scene()
    med = S.random_absorption_grid((9, 8, 10), LO, HI, seed=5, scale=1.5)
    img, tape = gs.render(medium=_gpu_medium(med))
    assert tape.stats["status"] == dt.DT_OK
    assert tape.stats["medium_samples"] > 0
    for v, excluded in enumerate([0.0531, 0.0719]):
        assert_radiance_parity(img[v], _oracle(gs, med, v), excluded)
    # the grid absorbs: darker than sigma alone wherever light crossed the object
    plain, ptape = gs.render()
    assert (img <= plain * (1 + 1e-5) + 1e-7).all() and (img < plain * 0.999).any()
    assert ptape.stats["medium_samples"] == 0


def test_constant_medium_equals_sigma_shift():
    gs = _scene(24, 20, depth=5)
    c = np.array([0.7, 0.2, 1.3], np.float32)
    med = dict(mu=np.broadcast_to(c, (3, 2, 4, 3)).copy(), lo=LO, hi=HI, step=0.05)
    img, _ = gs.render(medium=_gpu_medium(med))
    shifted = copy.copy(gs)
    shifted.sigma = gs.sigma + torch.from_numpy(c).cuda()
    ref, _ = shifted.render()
    np.testing.assert_allclose(img.cpu().numpy(), ref.cpu().numpy(), rtol=2e-5, atol=1e-6)


def _seed(gs, orc, rng, expected_excluded):
    g = rng.normal(size=(gs.cams.shape[0], gs.height, gs.width, 3))
    g[1:] = 0.0
    g[0][excluded_pixels(orc, expected_excluded)] = 0.0
    return g


def test_medium_gradients_match_oracle_derivative():
    """dJ/d(node values) along two random directions, dJ/dIoR and dJ/dsigma
    against the oracle's forward-mode derivative (view 0)."""
    gs = _scene(32, 28, depth=5)
    med = S.random_absorption_grid((6, 7, 5), LO, HI, seed=8, scale=1.2)
    rng = np.random.default_rng(41)
    orc = _oracle(gs, med)
    g = _seed(gs, orc, rng, 0.048)
    img, tape = gs.render(medium=_gpu_medium(med))
    dV, dior, dsig, dmu = dt.render_backward(tape, torch.from_numpy(g.astype(np.float32)).cuda())
    om = _oracle_medium(med)
    U = rng.normal(size=(2,) + om["mu"].shape)
    tmu = np.concatenate([np.zeros((4,) + om["mu"].shape), U])
    tior = np.array([1.0, 0, 0, 0, 0, 0])
    tsig = np.zeros((6, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    p = gs.params
    _, d = O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, None, tior, tsig,
                        p.spp, p.jitter, p.seed, 0, p.t_min, medium=om, tmu=tmu)
    J = np.einsum("khwc,hwc->k", d, g[0])
    assert float(dior) == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1.0, abs(J[0])))
    np.testing.assert_allclose(dsig.cpu().numpy(), J[1:4], rtol=GRAD_RTOL, atol=1e-6 * max(1.0, np.abs(J[1:4]).max()))
    dm = dmu.cpu().numpy().astype(np.float64)
    assert np.abs(dm).max() > 0
    for j in range(2):
        proj = float((dm * U[j]).sum())
        # |<e, u>| ~ |e| for u ~ N(0, I): bounded against the gradient's norm
        assert abs(proj - J[4 + j]) <= GRAD_RTOL * abs(J[4 + j]) + 3 * GRAD_RTOL * np.linalg.norm(dm), (proj, J[4 + j])


def test_medium_vertex_gradient_with_a_linear_field():
    """Moving a vertex moves every interior segment's length and samples; with
    a field linear in x the trilinear gradient has no jumps at cell faces, so
    the vertex gradient is smooth and compared along random directions."""
    gs = _scene(28, 24, views=1, depth=4, mesh="ico")
    b = np.array([[0.6, -0.3, 0.2], [0.1, 0.4, -0.5], [-0.2, 0.3, 0.7]])
    med = S.linear_absorption_grid((4, 5, 3), LO, HI, [0.9, 0.6, 1.1], b, 0.04)
    med["mu"] = med["mu"].astype(np.float32)
    rng = np.random.default_rng(43)
    orc = _oracle(gs, med)
    g = _seed(gs, orc, rng, 0.0223)
    img, tape = gs.render(medium=_gpu_medium(med))
    dV = dt.render_backward(tape, torch.from_numpy(g.astype(np.float32)).cuda())[0].cpu().numpy().astype(np.float64)
    nv = gs.Vn.shape[0]
    U = rng.normal(size=(2, nv, 3))
    p = gs.params
    _, d = O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, U, None, None,
                        p.spp, p.jitter, p.seed, 0, p.t_min, medium=_oracle_medium(med))
    J = np.einsum("khwc,hwc->k", d, g[0])
    for j in range(2):
        proj = float((dV * U[j]).sum())
        assert abs(proj - J[j]) <= GRAD_RTOL * abs(J[j]) + 3 * GRAD_RTOL * np.linalg.norm(dV), (proj, J[j])


def test_medium_in_a_batch_and_a_checkpointed_tape():
    """One batch holds a scene with a grid and one without: each image and
    gradient equals its own render; the checkpointed tape gives the full
    tape's gradients."""
    gs = _scene(24, 24, depth=5)
    med = S.random_absorption_grid((5, 6, 4), LO, HI, seed=9, scale=1.0)
    m = _gpu_medium(med)
    sc = S.glass_icosphere_scene(width=20, height=20)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 20, 20, 4)
    rng = np.random.default_rng(44)
    g0 = torch.from_numpy(rng.normal(size=(2, 24, 24, 3)).astype(np.float32)).cuda()
    g1 = torch.from_numpy(rng.normal(size=(1, 20, 20, 3)).astype(np.float32)).cuda()
    items = [dt.BatchItem(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 24, 24, gs.params, medium=m),
             dt.BatchItem(ico.V, ico.F, ico.bvh, ico.N, ico.ior, ico.sigma, ico.env, ico.cams, 20, 20, ico.params)]
    imgs, btape = dt.render_batch(items)
    out = dt.render_batch_backward(btape, [g0, g1])
    assert len(out[0]) == 4 and len(out[1]) == 3
    a, ta = gs.render(medium=m)
    ga = dt.render_backward(ta, g0)
    b, tb = ico.render()
    gb = dt.render_backward(tb, g1)
    np.testing.assert_allclose(imgs[0].cpu().numpy(), a.cpu().numpy(), rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(imgs[1].cpu().numpy(), b.cpu().numpy(), rtol=1e-5, atol=1e-7)
    for x, y in ((out[0][0], ga[0]), (out[0][3], ga[3]), (out[1][0], gb[0])):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-4 * max(np.linalg.norm(y), 1e-12)
    ck = copy.copy(gs)
    p = gs.params
    ck.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, checkpoint=True)
    c, tc = ck.render(medium=m)
    gc = dt.render_backward(tc, g0)
    np.testing.assert_allclose(c.cpu().numpy(), a.cpu().numpy(), rtol=1e-6, atol=1e-7)
    for x, y in ((gc[0], ga[0]), (gc[3], ga[3])):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-4 * max(np.linalg.norm(y), 1e-12)


def test_medium_arguments_are_checked():
    gs = _scene(8, 8, views=1, depth=2)
    mu = torch.zeros(3, 3, 3, 4, device="cuda")
    for bad in (dict(lo=(0, 0, 0), hi=(0, 1, 1), step=0.1), dict(lo=LO, hi=HI, step=0.0)):
        with pytest.raises(dt.DiffTransError):
            gs.render(medium=dt.Medium(mu, bad["lo"], bad["hi"], bad["step"]))
    with pytest.raises(ValueError):
        dt.Medium(torch.zeros(1, 3, 3, 4, device="cuda"), LO, HI, 0.1)
