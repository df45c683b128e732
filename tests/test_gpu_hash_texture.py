"""The absorption rate as a multi-resolution hash texture (Eq. 11 with
mu_t(x) = sigma + G(x), G the sum over levels of trilinear lattices whose
corners live in per-level tables, dense where a level fits its table and at
Instant-NGP's spatial hash otherwise).  The CUDA forward and adjoint against
the FP64 oracle: radiance, and the gradient with respect to the table
entries (along random directions, against the oracle's forward-mode
derivative), IoR and sigma; a one-level dense texture against the dense
grid it stores; the texture in a batch next to a dense grid and a scene
without either; the checkpointed tape; argument checks."""
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


def _gpu_texture(tex):
    table = torch.from_numpy(np.asarray(tex["table"], np.float32)).cuda()
    return dt.HashTexture(table, tex["res"], tex["lo"], tex["hi"], tex["step"])


def _oracle_texture(tex):
    """The texture as the device sees it: float32 entries, box and step (as
    doubles)."""
    return dict(table=np.asarray(tex["table"], np.float32).astype(np.float64), res=list(tex["res"]),
                lo=tuple(float(np.float32(x)) for x in tex["lo"]),
                hi=tuple(float(np.float32(x)) for x in tex["hi"]), step=float(np.float32(tex["step"])))


def _scene(w=40, h=32, views=2, depth=6, sigma=(0.2, 0.05, 0.1)):
    V, F = S.two_tori_mesh(36)
    return GpuScene(V, F, 1.5, np.array(sigma, np.float32), S.sh_env_map(64, 32, 1),
                    S.fibonacci_views(views, 3.0, w, h), w, h, depth, spp=1, jitter=0, seed=0)


def _oracle(gs, tex, view=0, probe=PROBE):
    p = gs.params
    return O.render(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[view], p.max_depth, p.spp, p.jitter,
                    p.seed, view, p.t_min, probe=probe, medium=_oracle_texture(tex))


def _texture(seed=5, levels=4, log2_table=10, n_min=4, n_max=24, scale=1.5):
    tex = S.random_hash_texture(levels, log2_table, n_min, n_max, LO, HI, seed=seed, scale=scale)
    # the finer levels overflow the table and are hashed
    assert any(r ** 3 > (1 << log2_table) for r in tex["res"]) and any(r ** 3 <= (1 << log2_table) for r in tex["res"])
    return tex


def test_hash_texture_render_matches_oracle():
    gs = _scene()
    tex = _texture()
    img, tape = gs.render(medium=_gpu_texture(tex))
    assert tape.stats["status"] == dt.DT_OK
    assert tape.stats["medium_samples"] > 0
    for v, excluded in enumerate([0.0508, 0.0727]):
        assert_radiance_parity(img[v], _oracle(gs, tex, v), excluded)
    plain, _ = gs.render()
    assert (img <= plain * (1 + 1e-5) + 1e-7).all() and (img < plain * 0.999).any()


def _seed(gs, orc, rng, expected_excluded):
    g = rng.normal(size=(gs.cams.shape[0], gs.height, gs.width, 3))
    g[1:] = 0.0
    g[0][excluded_pixels(orc, expected_excluded)] = 0.0
    return g


@pytest.mark.parametrize("moments", [False, True])
def test_hash_texture_gradients_match_oracle_derivative(moments):
    """dJ/d(table entries) along two random directions, dJ/dIoR and
    dJ/dsigma against the oracle's forward-mode derivative (view 0); with
    the full tape, and with the tape that keeps the medium's moments from
    the forward (tape_mode 2: the backward reads no table value)."""
    gs = _scene(32, 28, depth=5)
    if moments:
        p = gs.params
        gs.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, moments=True)
    tex = _texture(seed=8, levels=3, log2_table=9, n_min=5, n_max=14, scale=1.2)
    rng = np.random.default_rng(51)
    orc = _oracle(gs, tex)
    g = _seed(gs, orc, rng, 0.048)
    img, tape = gs.render(medium=_gpu_texture(tex))
    assert_radiance_parity(img[0], orc, 0.048)
    dV, dior, dsig, dtab = dt.render_backward(tape, torch.from_numpy(g.astype(np.float32)).cuda())
    assert tuple(dtab.shape) == tex["table"].shape
    ot = _oracle_texture(tex)
    U = rng.normal(size=(2,) + ot["table"].shape)
    tmu = np.concatenate([np.zeros((4,) + ot["table"].shape), U])
    tior = np.array([1.0, 0, 0, 0, 0, 0])
    tsig = np.zeros((6, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    p = gs.params
    _, d = O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, None, tior, tsig,
                        p.spp, p.jitter, p.seed, 0, p.t_min, medium=ot, tmu=tmu)
    J = np.einsum("khwc,hwc->k", d, g[0])
    assert float(dior) == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1.0, abs(J[0])))
    np.testing.assert_allclose(dsig.cpu().numpy(), J[1:4], rtol=GRAD_RTOL, atol=1e-6 * max(1.0, np.abs(J[1:4]).max()))
    dm = dtab.cpu().numpy().astype(np.float64)
    assert np.abs(dm).max() > 0
    for j in range(2):
        proj = float((dm * U[j]).sum())
        # |<e, u>| ~ |e| for u ~ N(0, I): bounded against the gradient's norm
        assert abs(proj - J[4 + j]) <= GRAD_RTOL * abs(J[4 + j]) + 3 * GRAD_RTOL * np.linalg.norm(dm), (proj, J[4 + j])


def test_one_dense_level_is_the_dense_grid():
    """A one-level texture whose lattice fits its table stores node (i, j, k)
    at (k n + j) n + i: holding a dense grid's node values there it renders
    the dense grid's image, and its table gradient is the grid's node
    gradient in the same order (the entries past n^3 get none)."""
    gs = _scene(28, 24, views=1, depth=5)
    n = 7
    med = S.random_absorption_grid((n, n, n), LO, HI, seed=12, scale=1.3)
    table = np.full((1, 512, 3), 0.0, np.float32)
    table[0, :n ** 3] = med["mu"].reshape(-1, 3)
    tex = dict(table=table, res=[n], lo=LO, hi=HI, step=med["step"])
    grid = dt.Medium(torch.from_numpy(med["mu"]).cuda(), LO, HI, med["step"])
    a, ta = gs.render(medium=grid)
    b, tb = gs.render(medium=_gpu_texture(tex))
    np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-6, atol=1e-8)
    assert ta.stats["medium_samples"] == tb.stats["medium_samples"]
    g = torch.from_numpy(np.random.default_rng(52).normal(size=tuple(a.shape)).astype(np.float32)).cuda()
    ga = dt.render_backward(ta, g)
    gb = dt.render_backward(tb, g)
    dgrid = ga[3].cpu().numpy().reshape(-1, 3).astype(np.float64)
    dtab = gb[3].cpu().numpy()[0].astype(np.float64)
    assert np.linalg.norm(dtab[:n ** 3] - dgrid) <= 1e-5 * np.linalg.norm(dgrid)
    assert not dtab[n ** 3:].any()
    for x, y in ((gb[0], ga[0]), (gb[1], ga[1]), (gb[2], ga[2])):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-5 * max(np.linalg.norm(y), 1e-12)


def test_hash_texture_in_a_batch_and_a_checkpointed_tape():
    """One batch holds a scene with a hash texture, one with a dense grid and
    one with neither: each image and gradient equals its own render; the
    checkpointed tape gives the full tape's gradients."""
    gs = _scene(24, 24, depth=5)
    tex = _gpu_texture(_texture(seed=9, levels=3, log2_table=8, n_min=3, n_max=12))
    med = S.random_absorption_grid((5, 6, 4), LO, HI, seed=9, scale=1.0)
    grid = dt.Medium(torch.from_numpy(med["mu"]).cuda(), med["lo"], med["hi"], med["step"])
    sc = S.glass_icosphere_scene(width=20, height=20)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 20, 20, 4)
    rng = np.random.default_rng(53)
    g0 = torch.from_numpy(rng.normal(size=(2, 24, 24, 3)).astype(np.float32)).cuda()
    g1 = torch.from_numpy(rng.normal(size=(1, 20, 20, 3)).astype(np.float32)).cuda()
    items = [dt.BatchItem(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 24, 24, gs.params, medium=tex),
             dt.BatchItem(ico.V, ico.F, ico.bvh, ico.N, ico.ior, ico.sigma, ico.env, ico.cams, 20, 20, ico.params,
                          medium=grid),
             dt.BatchItem(ico.V, ico.F, ico.bvh, ico.N, ico.ior, ico.sigma, ico.env, ico.cams, 20, 20, ico.params)]
    imgs, btape = dt.render_batch(items)
    out = dt.render_batch_backward(btape, [g0, g1, g1])
    assert len(out[0]) == 4 and len(out[1]) == 4 and len(out[2]) == 3
    a, ta = gs.render(medium=tex)
    ga = dt.render_backward(ta, g0)
    b, tb = ico.render(medium=grid)
    gb = dt.render_backward(tb, g1)
    c, tc = ico.render()
    gc = dt.render_backward(tc, g1)
    for x, y in ((imgs[0], a), (imgs[1], b), (imgs[2], c)):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=1e-5, atol=1e-7)
    for x, y in ((out[0][0], ga[0]), (out[0][3], ga[3]), (out[1][0], gb[0]), (out[1][3], gb[3]), (out[2][0], gc[0])):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-4 * max(np.linalg.norm(y), 1e-12)
    ck = copy.copy(gs)
    p = gs.params
    ck.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, checkpoint=True)
    d, td = ck.render(medium=tex)
    gd = dt.render_backward(td, g0)
    np.testing.assert_allclose(d.cpu().numpy(), a.cpu().numpy(), rtol=1e-6, atol=1e-7)
    for x, y in ((gd[0], ga[0]), (gd[3], ga[3])):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= 1e-4 * max(np.linalg.norm(y), 1e-12)


def test_hash_texture_arguments_are_checked():
    gs = _scene(8, 8, views=1, depth=2)
    table = torch.zeros(2, 64, 4, device="cuda")
    with pytest.raises(dt.DiffTransError):
        gs.render(medium=dt.HashTexture(table, [4, 8], LO, HI, 0.0))
    bad = dt.HashTexture(table, [4, 8], LO, HI, 0.1)
    bad.res = [4, 1]  # below the two nodes a level needs, past the binding's own check
    with pytest.raises(dt.DiffTransError):
        gs.render(medium=bad)
    for args in ((torch.zeros(2, 48, 4, device="cuda"), [4, 8]), (table, [4]), (table, [4, 1]),
                 (torch.zeros(17, 64, 4, device="cuda"), [4] * 17)):
        with pytest.raises(ValueError):
            dt.HashTexture(args[0], args[1], LO, HI, 0.1)


def test_moments_tape_equals_full_tape():
    """tape_mode 2 (the medium pass keeps S, dS/dt and the derivatives of S
    with respect to each interior segment's origin and direction) against
    the full tape: the same images and, up to rounding order, the same
    gradients of the vertices, IoR, sigma and the table or grid; alone and
    in a batch of a hash texture, a dense grid and a scene without either."""
    gs = _scene(24, 24, depth=6)
    tex = _gpu_texture(_texture(seed=10, levels=4, log2_table=9, n_min=3, n_max=16))
    med = S.random_absorption_grid((6, 5, 7), LO, HI, seed=10, scale=1.1)
    grid = dt.Medium(torch.from_numpy(med["mu"]).cuda(), med["lo"], med["hi"], med["step"])
    sc = S.glass_icosphere_scene(width=20, height=20)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 20, 20, 4)
    rng = np.random.default_rng(54)
    g0 = torch.from_numpy(rng.normal(size=(2, 24, 24, 3)).astype(np.float32)).cuda()
    g1 = torch.from_numpy(rng.normal(size=(1, 20, 20, 3)).astype(np.float32)).cuda()

    def with_moments(x):
        y = copy.copy(x)
        p = x.params
        y.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, moments=True)
        return y

    def close(x, y, tol):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - y) <= tol * max(np.linalg.norm(y), 1e-12)

    refs = []
    for scene, m, g in ((gs, tex, g0), (ico, grid, g1), (ico, None, g1)):
        a, ta = scene.render(medium=m)
        b, tb = with_moments(scene).render(medium=m)
        assert tb.ws.moments and not ta.ws.moments
        assert ta.stats["segments"] == tb.stats["segments"]
        assert ta.stats["medium_samples"] == tb.stats["medium_samples"]
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=2e-6, atol=1e-7)
        ga, gb = dt.render_backward(ta, g), dt.render_backward(tb, g)
        assert len(ga) == len(gb)
        for x, y in zip(gb, ga):
            close(x, y, 1e-5)
        refs.append((a, ga))
    p = gs.params
    items = [dt.BatchItem(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 24, 24,
                          dt.Params(p.max_depth, moments=True), medium=tex)]
    q = ico.params
    for m in (grid, None):
        items.append(dt.BatchItem(ico.V, ico.F, ico.bvh, ico.N, ico.ior, ico.sigma, ico.env, ico.cams, 20, 20,
                                  dt.Params(q.max_depth, moments=True), medium=m))
    imgs, btape = dt.render_batch(items)
    assert btape.ws.moments
    out = dt.render_batch_backward(btape, [g0, g1, g1])
    for img, grads, (a, ga) in zip(imgs, out, refs):
        np.testing.assert_allclose(img.cpu().numpy(), a.cpu().numpy(), rtol=1e-5, atol=1e-7)
        for x, y in zip(grads, ga):
            close(x, y, 1e-4)
    with pytest.raises(ValueError):
        dt.dump_segments(tb)
    with pytest.raises(ValueError):
        dt.Params(4, checkpoint=True, moments=True)
