"""GPU forward path vs the FP64 oracle, element by element, through the C ABI.

Hit triangle ids must agree bit for bit per (sample, heap node) and radiance
within 1e-4 relative, on every pixel whose oracle path has no degenerate
event (a hit or near miss within 1e-6 of an edge, a near tie, a TIR or
inside/outside decision within 1e-6 of its threshold)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import (GpuScene, assert_hit_id_parity, assert_radiance_parity, assert_tree_weights,
                            degenerate_pixels, step_parity)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_vertex_normals_match_oracle():
    for V, F in [S.icosphere(3), S.two_tori_mesh(40)]:
        Vt = torch.from_numpy(V).cuda()
        Ft = torch.from_numpy(F).cuda()
        N = dt.vertex_normals(Vt, Ft).cpu().numpy()
        No = O.vertex_normals(V, F)
        np.testing.assert_allclose(N, No, rtol=0, atol=2e-5)


def test_zero_area_faces_render_and_differentiate():
    """Faces of zero area (a repeated vertex) add nothing to the Eq. 13
    normals, are never hit (Moller-Trumbore's determinant is 0) and add no
    gradient: normals, image and gradients stay finite and match the oracle
    and the same mesh without them."""
    V, F = S.icosphere(3)
    Fd = np.concatenate([F, F[:40, [0, 0, 2]], F[40:80, [1, 2, 2]]]).astype(np.int32)
    env = S.sh_env_map(64, 32, 0)
    cam = S.camera((0.4, 0.7, 2.8), (0, 0, 0), (0, 1, 0), 45.0, 32, 32)
    sigma = np.array([0.5, 1.0, 1.5], np.float32)
    Vt = torch.from_numpy(V).cuda()
    N = dt.vertex_normals(Vt, torch.from_numpy(Fd).cuda())
    assert torch.isfinite(N).all()
    np.testing.assert_allclose(N.cpu().numpy(), O.vertex_normals(V, Fd), rtol=0, atol=2e-5)
    np.testing.assert_array_equal(N.cpu().numpy(), dt.vertex_normals(Vt, torch.from_numpy(F).cuda()).cpu().numpy())
    gd = GpuScene(V, Fd, 1.45, sigma, env, [cam], 32, 32, 4)
    g0 = GpuScene(V, F, 1.45, sigma, env, [cam], 32, 32, 4)
    img_d, tape_d = gd.render()
    img_0, tape_0 = g0.render()
    assert tape_d.stats["segments"] == tape_0.stats["segments"]
    np.testing.assert_allclose(img_d.cpu().numpy(), img_0.cpu().numpy(), rtol=1e-6, atol=1e-7)
    assert_radiance_parity(img_d[0], gd.oracle(0), 0.0186)
    g = torch.randn_like(img_d)
    dVd, diord, dsigd = dt.render_backward(tape_d, g)
    dV0, dior0, dsig0 = dt.render_backward(tape_0, g)
    assert torch.isfinite(dVd).all()
    np.testing.assert_allclose(dVd.cpu().numpy(), dV0.cpu().numpy(), rtol=1e-4, atol=1e-5)
    assert float(diord) == pytest.approx(float(dior0), rel=1e-4, abs=1e-6)


def test_vertex_normals_backward_matches_finite_differences():
    """<dN/dV u, w> by central differences of the (FP64) oracle normals."""
    V, F = S.icosphere(2)
    rng = np.random.default_rng(0)
    w = rng.normal(size=V.shape).astype(np.float32)
    u = rng.normal(size=V.shape)
    dV = dt.vertex_normals_backward(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda(),
                                    torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)
    h = 1e-6
    Vd = V.astype(np.float64)
    fd = ((O.vertex_normals(Vd + h * u, F) - O.vertex_normals(Vd - h * u, F)) / (2 * h) * w).sum()
    assert (dV * u).sum() == pytest.approx(fd, rel=1e-4)


def _random_rays(rng, m, inside_frac=0.5, radius=0.85):
    k = int(m * inside_frac)
    o = rng.uniform(-2.5, 2.5, size=(m, 3))
    dirs = rng.normal(size=(k, 3))
    o[:k] = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * rng.uniform(0, radius, size=(k, 1))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


@pytest.fixture(params=[0, 1], ids=["lbvh", "sah"])
def builder(request):
    old = dt.set_tuning(bvh_builder=request.param)
    yield request.param
    dt.set_tuning(**old)


def _same_centroid_mesh(rng, n=300):
    """n large triangles of random orientation sharing one centroid: the SAH
    builder finds no bin boundary and splits at the median."""
    V = []
    for _ in range(n):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        tri = np.array([[1, 0, 0], [-0.5, 0.866, 0], [-0.5, -0.866, 0]]) * rng.uniform(0.3, 1.0)
        V.append(tri @ q.T)
    V = np.concatenate(V).astype(np.float32)
    return V, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


@pytest.mark.parametrize("mesh", ["icosphere", "ico80", "tori", "blob", "box", "single", "same_centroid"])
def test_bvh_closest_hit_matches_brute_force(mesh, builder):
    rng = np.random.default_rng(1)
    if mesh == "icosphere":
        V, F = S.icosphere(3)
    elif mesh == "ico80":
        V, F = S.icosphere(1)
    elif mesh == "same_centroid":
        V, F = _same_centroid_mesh(rng)
    elif mesh == "tori":
        V, F = S.two_tori_mesh(40)
    elif mesh == "blob":
        V, F = S.mesh_from_field(S.random_blob_field(rng), 6000)
    elif mesh == "box":
        V, F = S.box_grid(3, (1.0, 1.0, 0.2))
    else:
        V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
        F = np.array([[0, 1, 2]], np.int32)
    o, d = _random_rays(rng, 3000)
    if mesh == "single":
        o = rng.uniform(-0.5, 1.0, size=(3000, 3)).astype(np.float32)
        o[:, 2] = rng.choice([-1.0, 1.0], size=3000)
        d = (np.stack([rng.uniform(0, 1, 3000), rng.uniform(0, 1, 3000), np.zeros(3000)], 1) - o)
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    src = rng.integers(-1, F.shape[0], size=o.shape[0]).astype(np.int32)
    Vt, Ft = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    bvh = dt.build_bvh(Vt, Ft)
    tri, tbb = dt.closest_hit(bvh, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                              torch.from_numpy(src).cuda(), 1e-5)
    tri, tbb = tri.cpu().numpy(), tbb.cpu().numpy()
    otri, ot, ob1, ob2, ofl = O.closest_hit(V, F, o.astype(np.float64), d.astype(np.float64), src, 1e-5)
    ok = (ofl & (O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE)) == 0
    assert ok.mean() > (0.8 if mesh == "same_centroid" else 0.95)
    np.testing.assert_array_equal(tri[ok], otri[ok])
    h = ok & (otri >= 0)
    assert h.sum() > 100 or mesh == "single"
    # FP32 Moller-Trumbore: t and the hit point carry relative error ~1e-7 |x|;
    # the barycentrics carry ~eps |s||e| / |det|, large for grazing rays, so
    # they are checked through the hit point they reconstruct
    np.testing.assert_allclose(tbb[h, 0], ot[h], rtol=2e-5, atol=1e-6)
    Vd = V.astype(np.float64)
    tri_v = Vd[F[otri[h]]]
    def point(b1, b2):
        return tri_v[:, 0] * (1 - b1 - b2)[:, None] + tri_v[:, 1] * b1[:, None] + tri_v[:, 2] * b2[:, None]
    err = np.linalg.norm(point(tbb[h, 1].astype(np.float64), tbb[h, 2].astype(np.float64)) - point(ob1[h], ob2[h]),
                         axis=1)
    assert err.max() < 2e-5, err.max()
    np.testing.assert_allclose(tbb[h, 1], ob1[h], atol=2e-4)
    np.testing.assert_allclose(tbb[h, 2], ob2[h], atol=2e-4)


def test_refit_tracks_moved_vertices(builder):
    rng = np.random.default_rng(2)
    V, F = S.two_tori_mesh(40)
    Vt, Ft = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    bvh = dt.build_bvh(Vt, Ft)
    V2 = (V.astype(np.float64) + rng.normal(0, 0.01, size=V.shape)).astype(np.float32)
    dt.refit_bvh(bvh, torch.from_numpy(V2).cuda(), Ft)
    o, d = _random_rays(rng, 2000, inside_frac=0.0)
    tri, _ = dt.closest_hit(bvh, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), None, 1e-5)
    otri, *_, ofl = O.closest_hit(V2, F, o, d, None, 1e-5)
    ok = (ofl & (O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE)) == 0
    np.testing.assert_array_equal(tri.cpu().numpy()[ok], otri[ok])


def _parity(gs, expected_excluded, view=0, expected_unstable=None):
    img, tape = gs.render()
    torch.cuda.synchronize()
    orc = gs.oracle(view, segments=True)
    info = assert_radiance_parity(img[view], orc, expected_excluded)
    si, sf = dt.dump_segments(tape)
    si, sf = si.cpu().numpy(), sf.cpu().numpy()
    npix = gs.width * gs.height
    spp = gs.params.spp
    lo, hi = view * npix * spp, (view + 1) * npix * spp
    sel = (si[:, 0] >= lo) & (si[:, 0] < hi)
    n = assert_hit_id_parity(si[sel], orc, spp, view_offset=lo)
    if expected_unstable is not None:
        assert_tree_weights(gs, view, si[sel], sf[sel], expected_unstable)
    # and every segment of the tape, one step at a time from its own FP32 inputs
    sit, sft = dt.dump_segments(tape)
    step_parity(sit, sft, torch.arange(sit.shape[0], device=sit.device), gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn,
                gs.params.max_depth, gs.params.t_min)
    return img, tape, orc, info, n


def test_render_glass_icosphere_matches_oracle():
    """The one-icosphere workload in full: subdivision 3, IoR 1.5, no
    absorption, 64x64 at pixel centres, depth 4, 64x32 SH environment."""
    gs = GpuScene.from_scene(S.glass_icosphere_scene())
    # measured: 69 of 4096 pixels excluded, 2.9 % of the segments weight-unstable
    img, tape, orc, info, n = _parity(gs, 0.0168, expected_unstable=0.0293)
    st = tape.stats
    oc = orc["counters"]
    bad = degenerate_pixels(orc)
    if bad.sum() == 0:
        assert st["segments"] == oc["segments"]
        assert st["hits"] == oc["hits"] and st["misses"] == oc["misses"]
        assert st["discarded"] == oc["discarded"] and st["tir"] == oc["tir"]


@pytest.mark.parametrize("depth,excluded,unstable", [(0, 0.0, 0.0), (1, 0.0073, 0.0103), (6, 0.0089, 0.0222)])
def test_render_absorbing_off_axis(depth, excluded, unstable):
    sc = S.glass_icosphere_scene(width=48, height=40)
    cam = S.camera((1.3, 0.9, 2.5), (0.05, -0.1, 0.0), (0, 1, 0), 50.0, 48, 40)
    gs = GpuScene(sc.V, sc.F, 1.45, np.array([0.5, 1.0, 1.5], np.float32), sc.env, [cam], 48, 40, depth)
    _parity(gs, excluded, expected_unstable=unstable)


def test_sah_and_lbvh_trees_find_the_same_hits():
    """The builders differ in speed only: every segment of a depth-8 genus-2
    render has the same hit triangle and flags through both trees, and the
    SAH tree needs fewer node visits."""
    V, F = S.two_tori_mesh(48)
    cams = S.fibonacci_views(2, 3.0, 64, 64)
    out = {}
    for b in (0, 1):
        old = dt.set_tuning(bvh_builder=b)
        try:
            gs = GpuScene(V, F, 1.5, np.array([0.3, 0.1, 0.05], np.float32), S.sh_env_map(64, 32, 1), cams, 64, 64, 8)
            img, tape = gs.render()
            si, sf = dt.dump_segments(tape)
            out[b] = (img.cpu().numpy(), tape.stats, si.cpu().numpy(), sf.cpu().numpy())
        finally:
            dt.set_tuning(**old)
    (ia, sa, sia, sfa), (ib, sb, sib, sfb) = out[0], out[1]
    assert sa["segments"] == sb["segments"] and sa["level_count"] == sb["level_count"]
    ka = np.lexsort((sia[:, 1], sia[:, 0]))
    kb = np.lexsort((sib[:, 1], sib[:, 0]))
    np.testing.assert_array_equal(sia[ka], sib[kb])
    np.testing.assert_array_equal(sfa[ka], sfb[kb])
    np.testing.assert_allclose(ib, ia, rtol=1e-6, atol=1e-7)
    assert sb["nodes_visited"] < 0.9 * sa["nodes_visited"], (sa["nodes_visited"], sb["nodes_visited"])


# fraction of the segments of each view of the jittered genus-2 test whose
# throughput or contribution is not stable under the oracle's tilt (measured
# with the oracle alone): internal reflections amplify the tilt along the path
UNSTABLE_G2 = [0.3311, 0.2836, 0.2326]


def test_render_genus2_multi_view_jittered():
    V, F = S.two_tori_mesh(36)
    env = S.sh_env_map(64, 32, 1)
    cams = S.fibonacci_views(3, 3.0, 40, 40)
    gs = GpuScene(V, F, 1.52, np.array([0.3, 0.1, 0.05], np.float32), env, cams, 40, 40, 8, spp=2, jitter=1,
                  seed=77)
    img, tape = gs.render()
    for v, excluded in enumerate([0.1131, 0.1875, 0.1781]):
        orc = gs.oracle(v, segments=True)
        assert_radiance_parity(img[v], orc, excluded)
        si, sf = dt.dump_segments(tape)
        si, sf = si.cpu().numpy(), sf.cpu().numpy()
        npix = 40 * 40 * 2
        sel = (si[:, 0] >= v * npix) & (si[:, 0] < (v + 1) * npix)
        assert_hit_id_parity(si[sel], orc, 2, view_offset=v * npix)
        assert_tree_weights(gs, v, si[sel], sf[sel], UNSTABLE_G2[v])
    sit, sft = dt.dump_segments(tape)
    info = step_parity(sit, sft, torch.arange(sit.shape[0], device=sit.device), gs.Vn, gs.Fn, gs.iorf, gs.sigman,
                       gs.envn, 8)
    assert info["checked_per_depth"][8] > 0, info


def test_all_miss_view_shows_environment():
    sc = S.glass_icosphere_scene(width=16, height=16)
    cam = S.camera((0.0, 0.0, 3.0), (0.0, 0.0, 6.0), (0, 1, 0), 45.0, 16, 16)  # looking away
    gs = GpuScene(sc.V, sc.F, 1.5, np.zeros(3, np.float32), sc.env, [cam], 16, 16, 4)
    img, tape = gs.render()
    o, d = O.camera_rays(cam)
    np.testing.assert_allclose(img[0].cpu().numpy().reshape(-1, 3), O.env_lookup(sc.env, d), rtol=1e-5, atol=1e-6)
    assert tape.stats["hits"] == 0 and tape.stats["segments"] == 256


def test_single_pixel_and_single_triangle():
    V = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    env = S.sh_env_map(16, 8, 3)
    cam = S.camera((0.1, 0.1, 2.0), (0.1, 0.1, 0.0), (0, 1, 0), 30.0, 1, 1)
    gs = GpuScene(V, F, 1.5, np.zeros(3, np.float32), env, [cam], 1, 1, 3)
    _parity(gs, 0.0, expected_unstable=0.0)


def test_arena_overflow_is_reported_and_retried():
    sc = S.glass_icosphere_scene(width=32, height=32)
    gs = GpuScene.from_scene(sc)
    small = dt.Workspace(32 * 32 + 10, gs.V.device)
    img_small, tape = dt.render(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 32, 32, gs.params,
                                ws=small, check=False)
    st = dt.read_stats(small)
    assert st["status"] == dt.DT_ERR_QUEUE_OVERFLOW
    assert st["seg_needed"] > small.capacity
    img, tape = dt.render(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 32, 32, gs.params,
                          ws=dt.Workspace(32 * 32 + 10, gs.V.device))
    assert tape.stats["status"] == dt.DT_OK and tape.ws.capacity > small.capacity
    assert_radiance_parity(img[0], gs.oracle(0), 0.0293)


def test_host_rejects_bad_arguments():
    sc = S.glass_icosphere_scene(width=8, height=8)
    gs = GpuScene.from_scene(sc)
    with pytest.raises(dt.DiffTransError):
        dt.render(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 8, 8, dt.Params(31))
    with pytest.raises(dt.DiffTransError):
        dt.render(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 8, 8, dt.Params(4, spp=0))
    with pytest.raises(dt.DiffTransError):
        dt.render(gs.V, gs.F, gs.bvh, gs.N, gs.ior, gs.sigma, gs.env, gs.cams, 8, 8, dt.Params(4),
                  ws=dt.Workspace(10, gs.V.device))
