"""Pins of the FP64 oracle to facts fixed by optics, geometry and calculus.

Each test checks the oracle against something other than itself: Fresnel's
sine/tangent laws (a different closed form from the one the oracle codes),
Snell's law and the reflection law as geometric facts, the critical and
Brewster angles, exact invariants of the ray tree (IoR 1 reproduces the
environment; R + T = 1 conserves energy), closed-form light paths through a
slab and a sphere, an independent ray/triangle intersection, and central
finite differences for the forward-mode derivatives.  A plausible slip in the
oracle (a dropped term, a wrong sign or index, a swapped eta) fails one.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_00413_gb300 import scenes as S


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _configs(rng, theta):
    """Incoming directions d at angle theta to the normal n (d . n = -cos)."""
    m = theta.size
    n = _unit(rng.normal(size=(m, 3)))
    t = _unit(np.cross(n, rng.normal(size=(m, 3))))
    d = -(np.cos(theta)[:, None] * n) + np.sin(theta)[:, None] * t
    return _unit(d), n


# ---------------------------------------------------------------------------
# Sec. 3.3: Eqs. 3-8 at one interface
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("eta1,eta2", [(1.0, 1.5), (1.0, 1.3), (1.5, 1.0), (1.7, 1.0), (1.0, 1.0 / 1.5)])
def test_fresnel_matches_sine_and_tangent_laws(eta1, eta2):
    """Fresnel's laws in angle form: Rs = sin^2(ti-tt)/sin^2(ti+tt),
    Rp = tan^2(ti-tt)/tan^2(ti+tt) (Hecht, Optics, Sec. 4.6)."""
    rng = np.random.default_rng(1)
    crit = math.asin(eta2 / eta1) if eta2 < eta1 else math.pi / 2
    th = rng.uniform(math.radians(1.0), min(math.radians(85.0), crit - 1e-3), size=200)
    d, n = _configs(rng, th)
    wr, wt, R, T, tir = O.interface(d, n, eta1, eta2)
    assert not tir.any()
    tt = np.arcsin(eta1 * np.sin(th) / eta2)
    Rs = np.sin(th - tt) ** 2 / np.sin(th + tt) ** 2
    Rp = np.tan(th - tt) ** 2 / np.tan(th + tt) ** 2
    np.testing.assert_allclose(R, 0.5 * (Rs + Rp), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(R + T, 1.0, rtol=0, atol=1e-15)
    assert (R >= 0).all() and (R <= 1).all()


@pytest.mark.parametrize("eta1,eta2", [(1.0, 1.5), (1.5, 1.0)])
def test_normal_incidence(eta1, eta2):
    """At normal incidence R = ((n1-n2)/(n1+n2))^2 = 0.04 for glass, and the
    refracted ray continues straight."""
    n = _unit(np.array([[0.3, -0.2, 0.9]]))
    wr, wt, R, T, tir = O.interface(-n, n, eta1, eta2)
    assert R[0] == pytest.approx(0.04, abs=1e-15)
    np.testing.assert_allclose(wt[0], -n[0], atol=1e-15)
    np.testing.assert_allclose(wr[0], n[0], atol=1e-15)


def test_brewster_angle_kills_p_polarisation():
    """At theta_B = atan(n2/n1) the p-term vanishes: R = Rs/2 exactly."""
    for eta1, eta2 in [(1.0, 1.5), (1.5, 1.0), (1.0, 1.33)]:
        th = math.atan(eta2 / eta1)
        d, n = _configs(np.random.default_rng(2), np.array([th]))
        _, _, R, _, _ = O.interface(d, n, eta1, eta2)
        tt = math.asin(eta1 * math.sin(th) / eta2)
        Rs = math.sin(th - tt) ** 2 / math.sin(th + tt) ** 2
        assert abs(th + tt - math.pi / 2) < 1e-12
        assert R[0] == pytest.approx(0.5 * Rs, rel=1e-12)


@pytest.mark.parametrize("eta1,eta2", [(1.0, 1.5), (1.5, 1.0), (1.3, 1.0)])
def test_snell_reflection_law_and_coplanarity(eta1, eta2):
    rng = np.random.default_rng(3)
    crit = math.asin(eta2 / eta1) if eta2 < eta1 else math.pi / 2
    th = rng.uniform(0.01, min(1.5, crit - 1e-3), size=300)
    d, n = _configs(rng, th)
    wr, wt, R, T, tir = O.interface(d, n, eta1, eta2)
    wi = -d
    # reflection: equal angles, unit length, wr + wi along n
    np.testing.assert_allclose(np.einsum("ij,ij->i", wr, n), np.einsum("ij,ij->i", wi, n), atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(wr, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(np.cross(wr + wi, n), axis=1), 0.0, atol=1e-14)
    # refraction: unit, crosses to the other side, coplanar, Snell
    np.testing.assert_allclose(np.linalg.norm(wt, axis=1), 1.0, atol=1e-14)
    assert (np.einsum("ij,ij->i", wt, n) < 0).all()
    np.testing.assert_allclose(np.einsum("ij,ij->i", np.cross(wi, n), wt), 0.0, atol=1e-14)
    sin_t = np.linalg.norm(np.cross(wt, n), axis=1)
    np.testing.assert_allclose(eta2 * sin_t, eta1 * np.sin(th), rtol=1e-12)


def test_total_internal_reflection_at_critical_angle():
    """Leaving glass (1.5 -> 1): theta_c = asin(1/1.5) = 41.81 deg; just below
    it both rays exist and R -> 1, just above only reflection with R = 1."""
    th_c = math.asin(1.0 / 1.5)
    assert math.degrees(th_c) == pytest.approx(41.8103149, abs=1e-6)
    below = np.array([th_c - 1e-4, th_c - 1e-7])
    above = np.array([th_c + 1e-7, th_c + 1e-2, 1.2])
    d, n = _configs(np.random.default_rng(4), below)
    _, wt, R, T, tir = O.interface(d, n, 1.5, 1.0)
    assert not tir.any()
    assert R[0] > 0.8 and R[1] > 0.99
    d, n = _configs(np.random.default_rng(5), above)
    _, wt, R, T, tir = O.interface(d, n, 1.5, 1.0)
    assert tir.all()
    np.testing.assert_array_equal(R, 1.0)
    np.testing.assert_array_equal(T, 0.0)


def test_fresnel_reciprocity_and_grazing():
    """R(n1 -> n2, theta_i) = R(n2 -> n1, theta_t) (Stokes relations), and
    R -> 1 at grazing incidence."""
    rng = np.random.default_rng(6)
    th = rng.uniform(0.05, 1.4, size=100)
    d, n = _configs(rng, th)
    _, wt, R, _, _ = O.interface(d, n, 1.0, 1.5)
    # reverse path: incoming along -wt from the other side with normal -n
    _, _, R2, _, tir = O.interface(-wt, -n, 1.5, 1.0)
    assert not tir.any()
    np.testing.assert_allclose(R2, R, rtol=1e-10)
    d, n = _configs(rng, np.array([math.pi / 2 - 1e-6]))
    _, _, R, _, _ = O.interface(d, n, 1.0, 1.5)
    assert R[0] > 0.9999


# ---------------------------------------------------------------------------
# Eq. 13: vertex normals
# ---------------------------------------------------------------------------
def test_vertex_normals_octahedron_closed_form():
    """Regular octahedron: four faces with unit normals (+-1,+-1,+-1)/sqrt3
    meet at (1,0,0), so N = (1/3) * (4/sqrt3, 0, 0)."""
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    F = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                F.append((sx, sy, sz))
    F = np.array(F, np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    N = O.vertex_normals(V, F)
    for i in range(6):
        np.testing.assert_allclose(N[i], V[i] * 4.0 / (3.0 * math.sqrt(3.0)), atol=1e-15)


def test_vertex_normals_icosahedron_closed_form():
    """Icosahedron: five faces per vertex, each at cos(alpha) = r_in / r_out
    = phi^2 / (sqrt3 * sqrt(phi * sqrt5)) to the vertex direction, so
    N_v = (5/3) cos(alpha) v_hat."""
    V, F = S.icosphere(0)
    V = V.astype(np.float64)
    V = V / np.linalg.norm(V, axis=1, keepdims=True)
    phi = (1 + math.sqrt(5)) / 2
    cos_a = phi ** 2 / (math.sqrt(3) * math.sqrt(phi * math.sqrt(5)))
    N = O.vertex_normals(V, F)
    np.testing.assert_allclose(N, V * (5.0 / 3.0) * cos_a, atol=2e-7)  # V came through float32


def test_vertex_normals_flat_grid_interior():
    """A vertex strictly inside a flat grid face touches six coplanar
    triangles: N = (6/3) n = 2 n."""
    V, F = S.box_grid(3)
    N = O.vertex_normals(V, F)
    V = V.astype(np.float64)
    interior = (np.abs(V) < 0.999).sum(axis=1) == 2
    assert interior.sum() == 6 * 4
    for i in np.nonzero(interior)[0]:
        n = np.where(np.abs(V[i]) > 0.999, np.sign(V[i]), 0.0)
        np.testing.assert_allclose(N[i], 2.0 * n, atol=1e-15)


# ---------------------------------------------------------------------------
# Sec. 3.4 step 2: closest hit, against an independent intersection
# ---------------------------------------------------------------------------
def _closest_hit_by_areas(V, F, o, d, t_min):
    """Plane intersection plus signed-area barycentrics, all triangles."""
    V = V.astype(np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    nn = np.einsum("ij,ij->i", n, n)
    out = []
    for oi, di in zip(o, d):
        den = n @ di
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.einsum("ij,ij->i", a - oi, n) / den
        p = oi + t[:, None] * di
        wa = np.einsum("ij,ij->i", np.cross(b - p, c - p), n) / nn
        wb = np.einsum("ij,ij->i", np.cross(c - p, a - p), n) / nn
        wc = 1.0 - wa - wb
        ok = (t > t_min) & (wa >= 0) & (wb >= 0) & (wc >= 0) & (den != 0)
        if not ok.any():
            out.append((-1, 0, 0, 0))
            continue
        idx = np.nonzero(ok)[0]
        k = idx[np.argmin(t[idx])]
        out.append((k, t[k], wb[k], wc[k]))
    return out


def test_closest_hit_matches_area_barycentrics():
    V, F = S.icosphere(2)
    rng = np.random.default_rng(7)
    m = 400
    o = rng.uniform(-2.5, 2.5, size=(m, 3))
    o[: m // 2] = _unit(rng.normal(size=(m // 2, 3))) * rng.uniform(0, 0.85, size=(m // 2, 1))
    d = _unit(rng.normal(size=(m, 3)))
    tri, t, b1, b2, fl = O.closest_hit(V, F, o, d, None, 1e-5)
    ref = _closest_hit_by_areas(V, F, o, d, 1e-5)
    checked = 0
    for i in range(m):
        if fl[i] & (O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE):
            continue
        checked += 1
        assert tri[i] == ref[i][0]
        if tri[i] >= 0:
            assert t[i] == pytest.approx(ref[i][1], rel=1e-10)
            assert b1[i] == pytest.approx(ref[i][2], abs=1e-10)
            assert b2[i] == pytest.approx(ref[i][3], abs=1e-10)
    assert checked > 0.95 * m
    assert (tri[: m // 2] >= 0).all()  # rays from inside a closed mesh always hit


def test_closest_hit_skips_source_and_respects_t_min():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]], np.float64)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    o = np.array([[0.2, 0.2, 0.0], [0.2, 0.2, 0.0], [0.2, 0.2, -1e-6]])
    d = np.array([[0, 0, 1.0], [0, 0, 1.0], [0, 0, 1.0]])
    tri, t, *_ = O.closest_hit(V, F, o, d, np.array([0, -1, -1]), 1e-5)
    assert list(tri) == [1, 1, 1]  # the start triangle is skipped / within t_min
    assert t[0] == pytest.approx(1.0)


# ---------------------------------------------------------------------------
# environment lookup
# ---------------------------------------------------------------------------
def test_env_lookup_texel_centres_midpoints_and_wrap():
    W, H = 16, 8
    rng = np.random.default_rng(8)
    env = rng.uniform(0.1, 2.0, size=(H, W, 3))
    TH, PH = S.texel_directions(W, H)
    dirs = np.stack([np.sin(TH) * np.cos(PH), np.cos(TH), np.sin(TH) * np.sin(PH)], -1).reshape(-1, 3)
    np.testing.assert_allclose(O.env_lookup(env, dirs), env.reshape(-1, 3), rtol=1e-12)
    # halfway between columns j and j+1 of row i: the average
    i, j = 3, 5
    th = (i + 0.5) / H * math.pi
    ph = (j + 1.0) / W * 2 * math.pi
    dd = np.array([[math.sin(th) * math.cos(ph), math.cos(th), math.sin(th) * math.sin(ph)]])
    np.testing.assert_allclose(O.env_lookup(env, dd)[0], 0.5 * (env[i, j] + env[i, j + 1]), rtol=1e-12)
    # phi = 0 (+x) sits halfway between the last and the first column
    dd = np.array([[math.sin(th), math.cos(th), 0.0]])
    np.testing.assert_allclose(O.env_lookup(env, dd)[0], 0.5 * (env[i, 0] + env[i, W - 1]), rtol=1e-12)
    # continuity across the seam
    eps = 1e-9
    a = O.env_lookup(env, np.array([[math.cos(eps), 0.0, math.sin(eps)]]))
    b = O.env_lookup(env, np.array([[math.cos(-eps), 0.0, math.sin(-eps)]]))
    np.testing.assert_allclose(a, b, atol=1e-7)
    # poles: clamped rows
    np.testing.assert_allclose(O.env_lookup(env, np.array([[0, 1.0, 0]]))[0],
                               O.env_lookup(env, np.array([[1e-12, 1.0, 0]]))[0], atol=1e-9)
    const = S.constant_env(W, H, (0.25, 0.5, 0.75))
    np.testing.assert_allclose(O.env_lookup(const, _unit(rng.normal(size=(50, 3)))),
                               np.tile([0.25, 0.5, 0.75], (50, 1)), rtol=1e-15)


# ---------------------------------------------------------------------------
# camera
# ---------------------------------------------------------------------------
def test_camera_geometry():
    cam = S.camera((1.0, 2.0, 3.0), (0.0, 0.5, 0.0), (0, 1, 0), 45.0, 65, 33)
    o, d = O.camera_rays(cam)
    fwd = _unit(np.array(cam.at) - np.array(cam.eye))
    right = _unit(np.cross(fwd, cam.up))
    up = np.cross(right, fwd)
    D = d.reshape(33, 65, 3)
    np.testing.assert_allclose(D[16, 32], fwd, atol=1e-15)          # centre pixel
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(o, np.tile(cam.eye, (o.shape[0], 1)))
    assert D[0, 32] @ up > 0 and D[-1, 32] @ up < 0                  # row 0 on top
    assert D[16, 0] @ right < 0 and D[16, -1] @ right > 0            # column 0 on the left
    # mirror symmetry of pixel centres about the optical axis
    np.testing.assert_allclose(D[0, 32] @ up, -(D[-1, 32] @ up), atol=1e-15)
    # the rows span the vertical field of view: angle between the first and
    # last row centres = 2 atan((1 - 1/H) tan(fov/2)) -> fov as H grows
    tall = S.camera((0, 0, 3.0), (0, 0, 0), (0, 1, 0), 45.0, 1, 4001)
    _, dt = O.camera_rays(tall)
    ang = math.acos(np.clip(dt[0] @ dt[-1], -1, 1))
    assert ang == pytest.approx(math.radians(45.0), abs=2e-4)


def test_jitter_offsets_are_uniform_and_deterministic():
    """The per-sample offsets (a counter-based PCG hash, a convention both
    sides implement) lie in [0,1)^2, look uniform, and repeat exactly."""
    cam = S.camera((0, 0, 3.0), width=32, height=32)
    o1, d1 = O.camera_rays(cam, spp=8, jitter=1, seed=123)
    o2, d2 = O.camera_rays(cam, spp=8, jitter=1, seed=123)
    _, d3 = O.camera_rays(cam, spp=8, jitter=1, seed=124)
    np.testing.assert_array_equal(d1, d2)
    assert not np.array_equal(d1, d3)
    _, dc = O.camera_rays(cam)
    # every jittered ray stays inside its pixel's footprint around the centre ray
    ang = np.arccos(np.clip(np.einsum("ij,ij->i", d1, np.repeat(dc, 8, axis=0)), -1, 1))
    pix = 2 * math.tan(math.radians(22.5)) / 32
    assert ang.max() < pix
    assert O.pcg_hash(0) != O.pcg_hash(1)
    vals = np.array([O.pcg_hash(i) >> 8 for i in range(20000)]) / 2.0 ** 24
    hist, _ = np.histogram(vals, bins=16, range=(0, 1))
    chi2 = ((hist - 1250.0) ** 2 / 1250.0).sum()
    assert chi2 < 40.0  # 15 dof, p ~ 5e-4


def test_pcg_hash_matches_values_worked_from_its_definition():
    """The PCG hash of Jarzynski & Olano (JCGT 2020): state = v * 747796405 +
    2891336453; word = ((state >> ((state >> 28) + 4)) ^ state) * 277803737;
    out = (word >> 22) ^ word, all modulo 2^32.  Values worked out step by
    step (hex):
      v = 0:          state ac564b05, shift 10 + 4 = 14, xor ac54fa5c,
                      word 07bb2ffc, out 07bb2fe2 = 129708002
      v = 1:          state d8e8c2ba, shift 13 + 4 = 17, xor d8e8aece,
                      word a8bee89e, out a8beea3c = 2831084092
      v = ffffffff:   state 7fc3d350, shift 7 + 4 = 11, xor 7fcc2b2a,
                      word e62a4a9a, out e62a4902 = 3861530882
      v = 3039 (12345): state 0f64e252, shift 0 + 4 = 4, xor 0f92ac77,
                      word f45eaedf, out f45ead0e = 4099845390
    A wrong multiplier, increment, shift or final xor changes every one."""
    assert O.pcg_hash(0) == 129708002
    assert O.pcg_hash(1) == 2831084092
    assert O.pcg_hash(0xFFFFFFFF) == 3861530882
    assert O.pcg_hash(12345) == 4099845390


def test_jitter_offset_matches_the_chained_hash_worked_by_hand():
    """The jitter of sample s of pixel p in view v with seed S chains the hash
    as h = pcg(pcg(pcg(pcg(S_lo ^ pcg(S_hi)) ^ v) ^ p) ^ s) and offsets the
    sample by ((pcg(h) >> 8) 2^-24, (pcg(h ^ 9e3779b9) >> 8) 2^-24) inside
    its pixel.  For S = 77, v = 2, p = 5, s = 1 (worked with the values of the
    hash above): pcg(0) = 07bb2fe2, 77 ^ that = 07bb2faf -> 86bc5bbc; ^ 2 ->
    7ac1f45f; ^ 5 -> bea75399; ^ 1 -> 9cad4b68 = h; pcg(h) = 308feb49 ->
    3182571 / 2^24 = 0.18969601392745972; pcg(h ^ 9e3779b9) = 2d5c41a1 ->
    2972737 / 2^24 = 0.1771889328956604.  The offset is read back from the
    oracle's jittered camera ray by inverting the pinhole projection."""
    W = H = 8
    cam = S.camera((0.3, -0.2, 3.0), (0.0, 0.1, 0.0), (0, 1, 0), 40.0, W, H)
    _, d = O.camera_rays(cam, spp=2, jitter=1, seed=77, view=2)
    ray = (0 * W + 5) * 2 + 1                     # pixel (5, 0), sample 1
    fwd = _unit(np.asarray(cam.at, float) - np.asarray(cam.eye, float))
    right = _unit(np.cross(fwd, cam.up))
    up = np.cross(right, fwd)
    th = math.tan(math.radians(cam.fov_y_deg) / 2)
    v = d[ray] / (d[ray] @ fwd)
    sx = ((v @ right) / (th * W / H) + 1.0) * W / 2  # px + jx
    sy = (1.0 - (v @ up) / th) * H / 2               # py + jy
    assert sx - 5 == pytest.approx(3182571 / 2.0 ** 24, abs=1e-9)
    assert sy - 0 == pytest.approx(2972737 / 2.0 ** 24, abs=1e-9)
    # 77 ^ pcg(0) worked above
    assert 77 ^ 0x07BB2FE2 == 0x07BB2FAF and O.pcg_hash(0x07BB2FAF) == 0x86BC5BBC
    assert O.pcg_hash(0x86BC5BBC ^ 2) == 0x7AC1F45F and O.pcg_hash(0x7AC1F45F ^ 5) == 0xBEA75399
    assert O.pcg_hash(0xBEA75399 ^ 1) == 0x9CAD4B68


# ---------------------------------------------------------------------------
# the whole ray tree (Sec. 3.4 steps 1-5)
# ---------------------------------------------------------------------------
def test_segment_throughputs_and_contributions():
    """The per-segment records of the tree (Sec. 3.4 steps 3-5): a camera
    ray starts with throughput 1; the children of a hit split its throughput
    W times the segment's absorption A by R + T = 1 (Eq. 8), so W_r + W_t =
    W A, with A = 1 outside and exp(-sigma t) inside, t the segment's own
    length; a TIR child takes all of it; an escaped segment contributes
    W * E(d); and a pixel's radiance is the sum of its escaped segments'
    contributions over its samples, divided by spp."""
    sc = S.glass_icosphere_scene(width=20, height=20)
    sigma = np.array([0.6, 0.25, 1.1])
    spp = 2
    r = O.render(sc.V, sc.F, 1.45, sigma, sc.env, sc.cams[0], 6, spp=spp, jitter=1, seed=3, segments=True)
    si, sf = r["seg_i"], r["seg_f"]
    rec = {(int(a), int(n)): j for j, (a, n, _, _) in enumerate(si)}
    roots = [j for (a, n), j in rec.items() if n == 1]
    np.testing.assert_array_equal(sf[roots, 9:12], 1.0)
    n_split = n_tir = 0
    for (a, n), j in rec.items():
        kids = [rec.get((a, 2 * n)), rec.get((a, 2 * n + 1))]
        if kids[0] is None:
            continue
        A = np.exp(-sigma * sf[j, 0]) if si[j, 3] & O.SEG_INSIDE else np.ones(3)
        W = sf[kids[0], 9:12] + (sf[kids[1], 9:12] if kids[1] is not None else 0.0)
        np.testing.assert_allclose(W, sf[j, 9:12] * A, rtol=1e-12)
        n_split += kids[1] is not None
        n_tir += kids[1] is None
    assert n_split > 100 and n_tir > 10
    miss = (si[:, 3] & O.SEG_MISS) != 0
    E = O.env_lookup(sc.env, sf[miss, 6:9])
    np.testing.assert_allclose(sf[miss, 12:15], sf[miss, 9:12] * E, rtol=1e-12)
    np.testing.assert_array_equal(sf[~miss, 12:15], 0.0)
    img = np.zeros((20 * 20, 3))
    np.add.at(img, si[:, 0] // spp, sf[:, 12:15] / spp)
    np.testing.assert_allclose(img, r["img"].reshape(-1, 3), rtol=1e-12, atol=1e-15)


def test_one_step_tracing_reproduces_the_tree():
    """trace_steps, fed every segment of a rendered tree (its origin,
    direction, depth and the triangle it leaves), returns that segment's hit
    and its children's directions and throughputs relative to its own: the
    tree of render() step by step (absorbing glass, depth 5, two jittered
    samples, TIR paths included)."""
    sc = S.glass_icosphere_scene(width=20, height=20)
    sigma = np.array([0.6, 0.25, 1.1])
    r = O.render(sc.V, sc.F, 1.45, sigma, sc.env, sc.cams[0], 5, spp=2, jitter=1, seed=3, segments=True)
    si, sf = r["seg_i"], r["seg_f"]
    rec = {(int(a), int(n)): j for j, (a, n, _, _) in enumerate(si)}
    src = np.array([si[rec[(a, n // 2)], 2] if n > 1 else -1 for a, n, _, _ in si])
    k = np.floor(np.log2(si[:, 1])).astype(int)
    ti, tf = O.trace_steps(sc.V, sc.F, 1.45, sigma, sc.env, sf[:, 3:6], sf[:, 6:9], src, k, 5)
    np.testing.assert_array_equal(ti[:, 0, 2], si[:, 2])
    np.testing.assert_array_equal(ti[:, 0, 3], si[:, 3])
    np.testing.assert_allclose(tf[:, 0, 12:15], sf[:, 12:15] / sf[:, 9:12], rtol=1e-12)
    n_kids = 0
    for j, (a, n, _, _) in enumerate(si):
        for c, node in ((1, 2 * n), (2, 2 * n + 1)):
            if (a, node) in rec:
                q = rec[(a, node)]
                assert ti[j, c, 1] == node - 2 * n + 2
                np.testing.assert_allclose(tf[j, c, 3:9], sf[q, 3:9], rtol=0, atol=1e-14)
                np.testing.assert_allclose(tf[j, c, 9:12] * sf[j, 9:12], sf[q, 9:12], rtol=1e-12)
                n_kids += 1
            else:
                assert ti[j, c, 1] == 0
    assert n_kids > 500


def test_ior_one_reproduces_environment_and_has_no_vertex_gradient():
    """IoR 1, no absorption: R = 0, T = 1, refraction is the identity, so
    every pixel shows E(d_camera) exactly and moving vertices changes nothing."""
    sc = S.glass_icosphere_scene(width=32, height=32)
    cam = sc.cams[0]
    r = O.render(sc.V, sc.F, 1.0, np.zeros(3), sc.env, cam, 4)
    _, d = O.camera_rays(cam)
    np.testing.assert_allclose(r["img"].reshape(-1, 3), O.env_lookup(sc.env, d), rtol=1e-12, atol=0)
    assert r["counters"]["hits"] > 0
    tV = np.random.default_rng(9).normal(size=(2,) + sc.V.shape)
    _, dimg = O.render_jvp(sc.V, sc.F, 1.0, np.zeros(3), sc.env, cam, 4, tV=tV)
    assert np.abs(dimg).max() < 1e-12


@pytest.mark.parametrize("which", ["icosphere", "blob"])
def test_energy_conservation_with_constant_environment(which):
    """No absorption and a constant environment E: every leaf of the tree is E
    or lost (depth limit, backfacing), and R + T = 1 splits weight exactly, so
    pixel = E * (1 - lost weight)."""
    if which == "icosphere":
        V, F = S.icosphere(3)
    else:
        V, F = S.mesh_from_field(S.random_blob_field(np.random.default_rng(10)), 1500)
    env = S.constant_env(8, 4, (0.3, 0.6, 0.9))
    E = env[0, 0].astype(np.float64)
    cam = S.camera((0.3, 0.8, 2.7), width=24, height=24)
    r = O.render(V, F, 1.5, np.zeros(3), env, cam, 6)
    np.testing.assert_allclose(r["img"], E * (1.0 - r["discard"]), rtol=1e-12, atol=1e-14)
    assert r["counters"]["discarded"] > 0


def _slab_series(ior, sigma, h, E, D):
    """Closed form for a slab at normal incidence: camera ray (depth 0) hits
    the front face; interior segments of length h alternate between faces,
    each hit reflecting R0 back inside and transmitting T0 out to E."""
    R0 = ((ior - 1.0) / (ior + 1.0)) ** 2
    T0 = 1.0 - R0
    A = np.exp(-np.asarray(sigma) * h)
    L_in = np.zeros(3)  # radiance of the interior segment at depth D: 0
    for k in range(D - 1, 0, -1):
        L_in = A * (R0 * L_in + T0 * E)
    return R0 * E + T0 * L_in


def _slab_scene(h):
    V, F = S.box_grid(3, (1.0, 1.0, h / 2))
    return V, F


@pytest.mark.parametrize("D", [1, 2, 5, 8])
def test_slab_normal_incidence_multiple_reflection_series(D):
    h = 0.4
    V, F = _slab_scene(h)
    sigma = np.array([0.3, 1.0, 2.0])
    env = S.constant_env(8, 4, (0.3, 0.6, 0.9))
    E = env[0, 0].astype(np.float64)
    cam = S.camera((0.1, 0.05, 3.0), (0.1, 0.05, 0.0), (0, 1, 0), 45.0, 1, 1)
    r = O.render(V, F, 1.5, sigma, env, cam, D, segments=True)
    expect = _slab_series(1.5, sigma, float(np.float32(h / 2)) * 2, E, D)
    np.testing.assert_allclose(r["img"][0, 0], expect, rtol=1e-12)
    inside = (r["seg_i"][:, 3] & O.SEG_INSIDE) != 0
    np.testing.assert_allclose(r["seg_f"][inside, 0], float(np.float32(h / 2)) * 2, rtol=1e-12)


def test_slab_derivatives_match_closed_form():
    """d(pixel)/d(sigma_c) and d(pixel)/d(IoR) of the slab series (central
    differences of the closed form) against the oracle's forward mode."""
    h, D = 0.4, 6
    V, F = _slab_scene(h)
    hh = float(np.float32(h / 2)) * 2
    sigma = np.array([0.3, 1.0, 2.0])
    env = S.constant_env(8, 4, (0.3, 0.6, 0.9))
    E = env[0, 0].astype(np.float64)
    cam = S.camera((0.1, 0.05, 3.0), (0.1, 0.05, 0.0), (0, 1, 0), 45.0, 1, 1)
    tsig = np.eye(3)
    tior = np.array([0.0, 0.0, 0.0, 1.0])
    tsig4 = np.vstack([tsig, np.zeros(3)])
    _, dimg = O.render_jvp(V, F, 1.5, sigma, env, cam, D, tior=tior, tsigma=tsig4)
    eps = 1e-6
    for c in range(3):
        sp, sm = sigma.copy(), sigma.copy()
        sp[c] += eps
        sm[c] -= eps
        fd = (_slab_series(1.5, sp, hh, E, D) - _slab_series(1.5, sm, hh, E, D)) / (2 * eps)
        np.testing.assert_allclose(dimg[c, 0, 0], fd, rtol=1e-7, atol=1e-12)
    fd = (_slab_series(1.5 + eps, sigma, hh, E, D) - _slab_series(1.5 - eps, sigma, hh, E, D)) / (2 * eps)
    np.testing.assert_allclose(dimg[3, 0, 0], fd, rtol=1e-7, atol=1e-12)


def test_slab_oblique_lateral_shift():
    """Oblique ray through a parallel slab: it leaves parallel to how it came
    in, shifted sideways by h sin(theta - theta_t) / cos(theta_t), after an
    interior path of length h / cos(theta_t)."""
    h, ior = 0.4, 1.5
    V, F = _slab_scene(h)
    hh = float(np.float32(h / 2)) * 2
    th = math.radians(30.0)
    d = np.array([[math.sin(th), 0.0, -math.cos(th)]])
    o = np.array([[-0.1 - (3.0 - hh / 2) * math.tan(th), 0.05, 3.0]])
    r = O.render_rays(V, F, ior, np.zeros(3), S.constant_env(8, 4, (1, 1, 1)), o, d, 3, segments=True)
    nodes = {int(n): i for i, n in enumerate(r["seg_i"][:, 1])}
    assert {1, 3, 7} <= set(nodes)
    assert r["seg_i"][nodes[7], 2] == -1          # the transmitted ray escapes
    sf = r["seg_f"]
    tt = math.asin(math.sin(th) / ior)
    np.testing.assert_allclose(sf[nodes[3], 0], hh / math.cos(tt), rtol=1e-12)
    d_out = sf[nodes[7], 6:9]
    np.testing.assert_allclose(d_out, d[0], atol=1e-14)
    x_out = sf[nodes[7], 3:6]
    off = x_out - o[0]
    shift = np.linalg.norm(off - (off @ d[0]) * d[0])
    assert shift == pytest.approx(hh * math.sin(th - tt) / math.cos(tt), rel=1e-11)


def test_sphere_refraction_converges_quadratically():
    """Rays parallel to -z at impact parameter b on a unit sphere:
    theta_i = asin(b), theta_t = asin(b / n); interior chord 2 cos(theta_t);
    deviation after two refractions 2 (theta_i - theta_t).  The icosphere's
    error must shrink about 4x per subdivision (faceting is O(h^2))."""
    ior = 1.5
    rng = np.random.default_rng(11)
    bs = np.array([0.3, 0.55, 0.7])
    az = rng.uniform(0, 2 * math.pi, size=bs.size)
    o = np.stack([bs * np.cos(az), bs * np.sin(az), np.full(bs.size, 3.0)], -1)
    d = np.tile([0.0, 0.0, -1.0], (bs.size, 1))
    errs = []
    for s in (3, 4, 5, 6):
        V, F = S.icosphere(s)
        r = O.render_rays(V, F, ior, np.zeros(3), S.constant_env(8, 4, (1, 1, 1)), o, d, 2, segments=True)
        e = 0.0
        for k in range(bs.size):
            m = r["seg_i"][:, 0] == k
            nodes = {int(n): i for i, n in zip(np.nonzero(m)[0], r["seg_i"][m, 1])}
            ti, tt = math.asin(bs[k]), math.asin(bs[k] / ior)
            chord = r["seg_f"][nodes[3], 0]
            dout = r["seg_f"][nodes[7], 6:9]
            dev = math.acos(np.clip(dout @ d[k], -1, 1))
            e = max(e, abs(chord - 2 * math.cos(tt)), abs(dev - 2 * (ti - tt)))
        errs.append(e)
    for a, b in zip(errs, errs[1:]):
        assert b < a / 2.5, errs
    assert errs[-1] < 2e-3


def test_forward_mode_matches_central_differences():
    """The dual-number derivative of the whole tree equals central finite
    differences of the value code, on pixels whose event signature (hit ids,
    inside/outside, TIR) is the same at +h and -h."""
    sc = S.glass_icosphere_scene(width=24, height=24)
    sigma = np.array([0.5, 1.0, 1.5])
    cam = sc.cams[0]
    rng = np.random.default_rng(12)
    tV = rng.normal(size=(1,) + sc.V.shape)
    _, dV = O.render_jvp(sc.V, sc.F, sc.ior, sigma, sc.env, cam, 4, tV=tV)
    _, dP = O.render_jvp(sc.V, sc.F, sc.ior, sigma, sc.env, cam, 4, tior=np.array([1.0, 0, 0]),
                         tsigma=np.array([[0, 0, 0], [1.0, 0, 0], [0, 0, 1.0]]))
    h = 1e-6
    V64 = sc.V.astype(np.float64)
    cases = [(V64 + h * tV[0], V64 - h * tV[0], sc.ior, sc.ior, sigma, sigma, dV[0])]
    cases.append((V64, V64, sc.ior + h, sc.ior - h, sigma, sigma, dP[0]))
    sp, sm = sigma.copy(), sigma.copy()
    sp[0] += h
    sm[0] -= h
    cases.append((V64, V64, sc.ior, sc.ior, sp, sm, dP[1]))
    for Vp, Vm, ip, im, sp_, sm_, jvp in cases:
        a = O.render(Vp, sc.F, ip, sp_, sc.env, cam, 4)
        b = O.render(Vm, sc.F, im, sm_, sc.env, cam, 4)
        stable = a["pix_sig"] == b["pix_sig"]
        assert stable.mean() > 0.9
        fd = (a["img"] - b["img"]) / (2 * h)
        scale = np.abs(jvp).max()
        assert scale > 0
        np.testing.assert_allclose(jvp[stable], fd[stable], rtol=0, atol=2e-6 * scale)


def test_zero_area_faces_add_nothing_to_vertex_normals():
    """Eq. 13 averages unit face normals; a face of zero area has none, so
    adding degenerate faces (a repeated vertex, three collinear vertices)
    leaves every vertex normal as it was and nothing becomes NaN."""
    V, F = S.icosphere(1)
    base = O.vertex_normals(V, F)
    m = V.shape[0]
    line = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [2.0, 0.0, 0.0]], V.dtype)  # exactly collinear
    V2 = np.concatenate([V, line])
    F2 = np.concatenate([F, [[F[0, 0], F[0, 0], F[0, 2]], [F[3, 1], F[3, 2], F[3, 2]], [m, m + 1, m + 2]]])
    n2 = O.vertex_normals(V2, F2.astype(np.int32))
    assert np.isfinite(n2).all()
    np.testing.assert_array_equal(n2[:m], base)
    np.testing.assert_array_equal(n2[m:], 0.0)


# ---------------------------------------------------------------------------
# Eq. 11 with a spatially varying absorption rate: a dense grid added to
# sigma on interior segments (trilinear, clamped to its box; steps of length
# h from the segment's start, the last one partial, sampled at midpoints)
# ---------------------------------------------------------------------------
def _segments_in_box(rng, n, lo, hi, t_max):
    """Random segments that stay inside [lo, hi]: start and end points drawn
    inside, t = their distance (capped at t_max by moving the end)."""
    lo, hi = np.asarray(lo), np.asarray(hi)
    a = lo + (hi - lo) * rng.uniform(0.05, 0.95, size=(n, 3))
    b = lo + (hi - lo) * rng.uniform(0.05, 0.95, size=(n, 3))
    d = _unit(b - a)
    t = np.minimum(np.linalg.norm(b - a, axis=1), t_max)
    return a, d, t


def test_medium_depth_of_a_linear_field_is_its_integral():
    """Trilinear interpolation reproduces a field linear in x exactly and the
    midpoint rule integrates a linear function exactly, so the optical depth
    is the closed form t (a + b . (o + d t / 2)) per channel, whatever the
    step (full steps, a partial last step, or a segment shorter than h)."""
    rng = np.random.default_rng(11)
    lo, hi = (-1.0, -0.8, -1.2), (1.1, 0.9, 1.0)
    a = np.array([0.3, 1.2, 0.05])
    b = rng.normal(size=(3, 3))
    for n, h in [((2, 2, 2), 0.1), ((5, 4, 6), 0.037), ((3, 7, 2), 1.5)]:
        med = S.linear_absorption_grid(n, lo, hi, a, b, h)
        o, d, t = _segments_in_box(rng, 200, lo, hi, 2.0)
        got = O.medium_depth(med, o, d, t)
        mid = o + d * (t / 2)[:, None]
        want = t[:, None] * (a[None, :] + mid @ b.T)
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)


def test_medium_depth_midpoint_error_of_a_bilinear_field():
    """mu = x y is reproduced exactly by trilinear interpolation; along a
    segment from the origin it is (dx dy) s^2, for which the midpoint rule
    over steps h_i errs by exactly -(dx dy) sum h_i^3 / 12.  With m full
    steps of length h and a last one of length r = t - m h this pins the
    step layout: t^3/3 - (m h^3 + r^3)/12, times dx dy."""
    rng = np.random.default_rng(12)
    lo, hi = (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0)
    X, Y, Z = S.grid_nodes((3, 3, 3), lo, hi)
    mu = np.stack([X * Y, 2.0 * X * Y, -X * Y], axis=-1)
    for h in (0.05, 0.13, 0.7):
        med = dict(mu=mu, lo=lo, hi=hi, step=h)
        d = _unit(rng.normal(size=(50, 3)))
        t = rng.uniform(0.01, 1.9, size=50)
        o = np.zeros((50, 3))
        got = O.medium_depth(med, o, d, t)
        m = np.floor(t / h)
        r = t - m * h
        base = d[:, 0] * d[:, 1] * (t ** 3 / 3.0 - (m * h ** 3 + r ** 3) / 12.0)
        np.testing.assert_allclose(got, base[:, None] * np.array([1.0, 2.0, -1.0]), rtol=1e-10, atol=1e-13)


def test_medium_is_clamped_to_its_box():
    """Beyond the box each clamped coordinate sees the boundary value: a
    field linear in x read past hi_x is the constant a + b hi_x."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    b = np.zeros((3, 3))
    b[:, 0] = [0.5, 1.0, 2.0]
    med = S.linear_absorption_grid((4, 3, 5), lo, hi, [0.1, 0.2, 0.3], b, 0.05)
    o = np.array([[1.5, 0.2, -0.3], [3.0, -2.0, 5.0]])
    d = _unit(np.array([[1.0, 0.3, 0.2], [0.2, -1.0, 0.1]]))
    t = np.array([0.8, 1.3])
    got = O.medium_depth(med, o, d, t)
    want = t[:, None] * (np.array([0.1, 0.2, 0.3]) + b[:, 0] * 1.0)[None, :]
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_medium_depth_is_continuous_across_step_boundaries():
    """The partial last step makes the sum continuous in t: just below and
    just above a multiple of h it differs by O(epsilon)."""
    med = S.random_absorption_grid((6, 5, 7), (-1.2, -1.2, -1.2), (1.2, 1.2, 1.2), seed=3)
    med["mu"] = med["mu"].astype(np.float64)
    h = med["step"]
    o = np.array([[-0.5, 0.1, 0.2]] * 2)
    d = _unit(np.array([[0.8, 0.3, -0.2]] * 2))
    for k in (1, 3, 7):
        eps = 1e-9
        got = O.medium_depth(med, o, d, np.array([k * h - eps, k * h + eps]))
        assert np.abs(got[1] - got[0]).max() < 1e-7


def test_constant_medium_is_a_sigma_shift():
    """A grid of constant node values c adds c t to the optical depth of
    every interior segment: the render equals the one with sigma + c."""
    sc = S.glass_icosphere_scene(width=12, height=10, max_depth=5)
    cam = sc.cams[0]
    sigma = np.array([0.2, 0.1, 0.4])
    c = np.array([0.5, 0.05, 1.1])
    mu = np.broadcast_to(c, (3, 4, 2, 3)).copy()
    med = dict(mu=mu, lo=(-1.5, -1.5, -1.5), hi=(1.5, 1.5, 1.5), step=0.07)
    a = O.render(sc.V, sc.F, 1.5, sigma, sc.env, cam, 5, medium=med)
    b = O.render(sc.V, sc.F, 1.5, sigma + c, sc.env, cam, 5)
    np.testing.assert_allclose(a["img"], b["img"], rtol=1e-11, atol=1e-14)
    assert a["counters"] == b["counters"]


def test_medium_jvp_matches_central_differences():
    """Forward-mode derivatives with respect to the grid's node values (and
    the vertices, whose moves change every interior segment's length and
    sample positions) against central differences of the FP64 render."""
    sc = S.glass_icosphere_scene(width=8, height=8, max_depth=4)
    cam = sc.cams[0]
    sigma = np.array([0.1, 0.2, 0.3])
    med = S.random_absorption_grid((4, 5, 3), (-1.1, -1.1, -1.1), (1.1, 1.1, 1.1), seed=7, scale=0.8)
    med["mu"] = med["mu"].astype(np.float64)
    rng = np.random.default_rng(13)
    tmu = rng.normal(size=(1,) + med["mu"].shape)
    tV = 0.01 * rng.normal(size=(1,) + sc.V.shape)
    V = sc.V.astype(np.float64)
    _, dm = O.render_jvp(V, sc.F, 1.5, sigma, sc.env, cam, 4, medium=med, tmu=tmu)
    _, dv = O.render_jvp(V, sc.F, 1.5, sigma, sc.env, cam, 4, tV=tV, medium=med)
    eps = 1e-6

    def img(mu=None, VV=V):
        m = dict(med, mu=med["mu"] if mu is None else mu)
        return O.render(VV, sc.F, 1.5, sigma, sc.env, cam, 4, medium=m)["img"]

    fd_m = (img(med["mu"] + eps * tmu[0]) - img(med["mu"] - eps * tmu[0])) / (2 * eps)
    fd_v = (img(VV=V + eps * tV[0]) - img(VV=V - eps * tV[0])) / (2 * eps)
    np.testing.assert_allclose(dm[0], fd_m, rtol=1e-5, atol=1e-8)
    # a vertex move can shift a sample across a cell face (where the
    # trilinear gradient jumps) only on a set of measure zero; compare
    # pixelwise with a small absolute floor
    np.testing.assert_allclose(dv[0], fd_v, rtol=1e-4, atol=1e-6)
    assert np.abs(dm[0]).max() > 1e-3 and np.abs(dv[0]).max() > 1e-3


def _point_values(med, P):
    """G at points P ([n, 3]) from the optical depth of a segment of length
    t = 2^-10 centred on each point with one (partial) step: S = G(p) t,
    exact in binary arithmetic for the points used here."""
    t = 2.0 ** -10
    d = np.tile([1.0, 0.0, 0.0], (len(P), 1))
    o = np.asarray(P, np.float64) - d * (t / 2)
    return O.medium_depth(dict(med, step=1.0), o, d, np.full(len(P), t)) / t


def test_hash_texture_of_dense_levels_reproduces_a_linear_field():
    """Levels with n^3 <= T index their nodes densely, (k n + j) n + i in
    their own slice [l T, (l + 1) T) of the table.  With level l holding
    the linear field a_l + b_l . x at its nodes (and garbage in the entries
    it does not use) the texture is the linear field sum_l a_l + b_l . x,
    whose optical depth is the closed form of the dense-grid pin."""
    rng = np.random.default_rng(21)
    lo, hi = (-1.0, -0.7, -1.3), (0.9, 1.2, 1.1)
    T, res = 512, [2, 5, 8]
    table = np.full((3, T, 3), 1e6)
    a_sum, b_sum = np.zeros(3), np.zeros((3, 3))
    for l, n in enumerate(res):
        a, b = rng.normal(size=3), rng.normal(size=(3, 3))
        lev = S.linear_absorption_grid((n, n, n), lo, hi, a, b, 0.1)["mu"]  # [n, n, n, 3], x fastest
        table[l, :n ** 3] = lev.reshape(-1, 3)
        a_sum, b_sum = a_sum + a, b_sum + b
    for h in (0.043, 0.31):
        med = dict(table=table, res=res, lo=lo, hi=hi, step=h)
        o, d, t = _segments_in_box(rng, 150, lo, hi, 2.0)
        got = O.medium_depth(med, o, d, t)
        want = t[:, None] * (a_sum[None, :] + (o + d * (t / 2)[:, None]) @ b_sum.T)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-11)


def test_hash_texture_hashed_level_reads_the_spatial_hash():
    """A level with n^3 > T stores corner (i, j, k) at (i XOR 2654435761 j
    XOR 805459861 k) mod T (Instant-NGP, Eq. 4).  With T = 64 only the low
    six bits of the products count: 2654435761 = 0x9E3779B1 = 49 and
    805459861 = 0x30025795 = 21 (mod 64), so by hand (5,0,0) -> 5,
    (0,1,0) -> 49, (0,0,1) -> 21, (1,1,0) -> 1^49 = 48, (1,1,1) -> 1^49^21
    = 37, (0,2,0) -> 98 mod 64 = 34, (3,5,7) -> 3^53^19 = 37, (8,8,8) ->
    8^8^40 = 40, (2,0,3) -> 2^63 = 61.  A table holding its own entry index
    (times 1, 2, -1 per channel) returns these at the lattice points (the
    box [0, 8]^3 with 9 nodes puts node (i, j, k) at (i, j, k)), and the
    mean of the two corners halfway between (0,1,0) and (1,1,0)."""
    T = 64
    e = np.arange(T, dtype=np.float64)
    med = dict(table=np.stack([e, 2 * e, -e], axis=-1)[None], res=[9], lo=(0.0, 0.0, 0.0), hi=(8.0, 8.0, 8.0))
    pts = [(5, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1), (0, 2, 0), (3, 5, 7), (8, 8, 8), (2, 0, 3),
           (0.5, 1, 0)]
    want = np.array([5, 49, 21, 48, 37, 34, 37, 40, 61, 48.5])
    got = _point_values(med, np.array(pts, np.float64))
    np.testing.assert_array_equal(got, want[:, None] * np.array([1.0, 2.0, -1.0]))


def test_hash_texture_levels_superpose():
    """The texture is the sum of its levels: a dense, a dense and a hashed
    level together give the sum of the three one-level textures' optical
    depths (each with its own table slice and node count)."""
    rng = np.random.default_rng(22)
    lo, hi = (-1.2, -1.1, -1.0), (1.0, 1.3, 1.1)
    med = S.random_hash_texture(3, 9, 4, 16, lo, hi, seed=5, scale=1.3)
    assert med["res"] == [4, 8, 16] and 16 ** 3 > 512 >= 8 ** 3
    med["table"] = med["table"].astype(np.float64)
    o, d, t = _segments_in_box(rng, 100, lo, hi, 2.0)
    got = O.medium_depth(med, o, d, t)
    parts = sum(O.medium_depth(dict(med, table=med["table"][l:l + 1], res=[med["res"][l]]), o, d, t)
                for l in range(3))
    np.testing.assert_allclose(got, parts, rtol=1e-12, atol=1e-13)
    assert np.abs(got).min() > 0


def test_constant_hash_texture_is_a_sigma_shift():
    """Every entry of every level c / L: the texture is the constant c (the
    trilinear weights sum to one at each level), so the render equals the
    one with sigma + c."""
    sc = S.glass_icosphere_scene(width=12, height=10, max_depth=5)
    cam = sc.cams[0]
    sigma = np.array([0.2, 0.1, 0.4])
    c = np.array([0.5, 0.05, 1.1])
    table = np.broadcast_to(c / 4.0, (4, 64, 3)).copy()
    med = dict(table=table, res=[2, 3, 5, 9], lo=(-1.5, -1.5, -1.5), hi=(1.5, 1.5, 1.5), step=0.07)
    a = O.render(sc.V, sc.F, 1.5, sigma, sc.env, cam, 5, medium=med)
    b = O.render(sc.V, sc.F, 1.5, sigma + c, sc.env, cam, 5)
    np.testing.assert_allclose(a["img"], b["img"], rtol=1e-11, atol=1e-14)
    assert a["counters"] == b["counters"]


def test_hash_texture_jvp_matches_central_differences():
    """Forward-mode derivatives with respect to the table entries (hashed
    collisions included) against central differences of the FP64 render."""
    sc = S.glass_icosphere_scene(width=8, height=8, max_depth=4)
    cam = sc.cams[0]
    sigma = np.array([0.1, 0.2, 0.3])
    med = S.random_hash_texture(3, 6, 3, 9, (-1.1, -1.1, -1.1), (1.1, 1.1, 1.1), seed=8, scale=0.8)
    med["table"] = med["table"].astype(np.float64)
    rng = np.random.default_rng(23)
    tmu = rng.normal(size=(1,) + med["table"].shape)
    V = sc.V.astype(np.float64)
    _, dm = O.render_jvp(V, sc.F, 1.5, sigma, sc.env, cam, 4, medium=med, tmu=tmu)
    eps = 1e-6

    def img(tab):
        return O.render(V, sc.F, 1.5, sigma, sc.env, cam, 4, medium=dict(med, table=tab))["img"]

    fd = (img(med["table"] + eps * tmu[0]) - img(med["table"] - eps * tmu[0])) / (2 * eps)
    np.testing.assert_allclose(dm[0], fd, rtol=1e-5, atol=1e-8)
    assert np.abs(dm[0]).max() > 1e-3


def test_field_corners_are_the_renderers_field():
    """The oracle's linear map of the field (entries and trilinear weights of
    each level's cell) reproduces the field the optical-depth sum samples:
    G at lattice-aligned points read through a one-step segment (the path
    the renderer takes) equals sum_k w_k values[idx_k]; every level's eight
    weights form a partition of unity, and points past the box read the
    boundary."""
    rng = np.random.default_rng(31)
    lo, hi = (0.0, 0.0, 0.0), (8.0, 8.0, 8.0)
    for med in (S.random_hash_texture(3, 6, 3, 9, lo, hi, seed=2),
                dict(mu=rng.uniform(size=(6, 4, 5, 3)), lo=lo, hi=hi, step=0.1)):
        key = "table" if "table" in med else "mu"
        med[key] = med[key].astype(np.float64)
        flat = med[key].reshape(-1, 3)
        x = rng.uniform(-1.0, 9.0, size=(200, 3))
        idx, w = O.field_corners(med, x)
        G = (w[..., None] * flat[idx]).sum(axis=1)
        np.testing.assert_allclose(O.field_eval(med, x), G, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(w.reshape(len(x), -1, 8).sum(axis=2), 1.0, atol=1e-14)
        assert (w >= 0).all() and idx.min() >= 0 and idx.max() < len(flat)
        pts = np.array([[1.0, 2.0, 3.0], [8.0, 0.0, 5.0], [4.0, 4.0, 4.0]])
        np.testing.assert_allclose(_point_values(med, pts), O.field_eval(med, pts), rtol=1e-12, atol=1e-14)
        far = np.array([[12.0, 3.0, -4.0]])
        np.testing.assert_allclose(O.field_eval(med, far), O.field_eval(med, [[8.0, 3.0, 0.0]]), rtol=1e-14)


def test_mat_smooth_loss_of_a_linear_field_is_closed_form():
    """Eq. 16 on a field linear in x, a + B x (reproduced exactly by a dense
    grid and by dense hash levels): mu_t(v) - mu_t(v + xi) = -B xi, so the
    loss is (1/N) sum_i ||B xi_i||_1 for points and perturbations inside the
    box; a zero perturbation and a constant field give 0 with no gradient."""
    rng = np.random.default_rng(32)
    lo, hi = (-1.0, -1.2, -0.9), (1.1, 1.0, 1.3)
    a, B = rng.normal(size=3), rng.normal(size=(3, 3))
    grid = S.linear_absorption_grid((4, 5, 3), lo, hi, a, B, 0.1)
    table = np.full((2, 512, 3), 7.0)
    for l, n in enumerate((3, 8)):
        table[l, :n ** 3] = S.linear_absorption_grid((n, n, n), lo, hi, a / 2, B / 2, 0.1)["mu"].reshape(-1, 3)
    tex = dict(table=table, res=[3, 8], lo=lo, hi=hi, step=0.1)
    v = np.asarray(lo) + 0.1 + (np.asarray(hi) - np.asarray(lo) - 0.2) * rng.uniform(size=(300, 3))
    xi = 0.05 * rng.normal(size=(300, 3))
    xi = np.clip(v + xi, np.asarray(lo), np.asarray(hi)) - v
    want = np.abs(xi @ B.T).sum() / 300
    for med in (grid, tex):
        loss, g = O.mat_smooth_loss(med, v, xi)
        assert loss == pytest.approx(want, rel=1e-11)
        assert g.shape == (med["table"] if "table" in med else med["mu"]).shape
        loss0, g0 = O.mat_smooth_loss(med, v, np.zeros_like(v))
        assert loss0 == 0.0 and not g0.any()
    const = dict(grid, mu=np.broadcast_to([0.3, 0.1, 0.2], grid["mu"].shape).copy())
    loss, g = O.mat_smooth_loss(const, v, xi)
    assert loss < 1e-14


def test_mat_smooth_gradient_matches_central_differences():
    """The loss is piecewise linear in the values: away from a channel
    difference of zero, central differences along a random direction of
    the table match the gradient (hashed levels included)."""
    rng = np.random.default_rng(33)
    tex = S.random_hash_texture(3, 6, 3, 9, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), seed=4)
    tex["table"] = tex["table"].astype(np.float64)
    v = rng.uniform(-1.0, 1.0, size=(80, 3))
    xi = 0.1 * rng.normal(size=(80, 3))
    loss, g = O.mat_smooth_loss(tex, v, xi)
    for _ in range(3):
        u = rng.normal(size=tex["table"].shape)
        eps = 1e-7
        lp = O.mat_smooth_loss(dict(tex, table=tex["table"] + eps * u), v, xi)[0]
        lm = O.mat_smooth_loss(dict(tex, table=tex["table"] - eps * u), v, xi)[0]
        assert (lp - lm) / (2 * eps) == pytest.approx(float((g * u).sum()), rel=1e-6)


def test_image_is_linear_in_the_environment():
    """Escaped radiance is read from the map and weighted by a throughput
    that does not depend on it (Sec. 3.4 steps 3-5), so the image is linear
    in the texels: render(a E1 + b E2) = a render(E1) + b render(E2).  (This
    is what makes render(env = u) the directional derivative of the image
    along u, the reference for the environment gradient.)"""
    sc = S.glass_icosphere_scene(width=10, height=8, max_depth=4)
    cam = sc.cams[0]
    sigma = np.array([0.3, 0.1, 0.2])
    rng = np.random.default_rng(17)
    E1, E2 = rng.normal(size=(2,) + sc.env.shape)
    a, b = 0.7, -1.3
    r = lambda E: O.render(sc.V, sc.F, 1.5, sigma, E, cam, 4)["img"]
    np.testing.assert_allclose(r(a * E1 + b * E2), a * r(E1) + b * r(E2), rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# Eqs. 14-15: the tracer stage's colour and tone losses
# ---------------------------------------------------------------------------
def test_paper_losses_closed_forms():
    """At c_hat = c both losses have zero gradient, L_color = 0 and
    L_tone = -mean var(c); at c_hat = k c (k > 0) the tone is exact (cosine
    1) and L_color = (k - 1)^2 mean sum c^4; for orthogonal colours the
    cosine is 0 and the tone term is 1 - var(c)."""
    rng = np.random.default_rng(61)
    c = rng.uniform(0.05, 1.0, size=(50, 3))
    var = c.var(axis=1)
    t, lc, lt, g = O.paper_losses(c, c, 0.7, 1.3)
    assert lc == 0.0 and lt == pytest.approx(-var.mean(), rel=1e-12) and np.abs(g).max() < 1e-15
    t, lc, lt, g = O.paper_losses(2.5 * c, c, 1.0, 1.0)
    assert lc == pytest.approx(1.5 ** 2 * (c ** 4).sum(axis=1).mean(), rel=1e-12)
    assert lt == pytest.approx(-var.mean(), rel=1e-12)
    a = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    b = np.array([[0.0, 3.0, 0.0], [0.0, 0.0, 0.5]])
    _, _, lt, _ = O.paper_losses(a, b, 1.0, 1.0)
    assert lt == pytest.approx(np.mean(1.0 - b.var(axis=1)), rel=1e-12)


def test_paper_losses_gradient_matches_central_differences():
    rng = np.random.default_rng(62)
    ch = rng.uniform(0.0, 1.2, size=(4, 5, 3))
    c = rng.uniform(0.05, 1.0, size=(4, 5, 3))
    _, _, _, g = O.paper_losses(ch, c, 0.8, 1.7)
    eps = 1e-6
    fd = np.zeros_like(ch)
    for idx in np.ndindex(ch.shape):
        p, m = ch.copy(), ch.copy()
        p[idx] += eps
        m[idx] -= eps
        fd[idx] = (O.paper_losses(p, c, 0.8, 1.7)[0] - O.paper_losses(m, c, 0.8, 1.7)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------------------
# the step after the gradient (App. A): Laplacian, large-steps solve,
# AdamUniform, L_edge
# ---------------------------------------------------------------------------
from oracle import mesh_update as MU  # noqa: E402


def _octahedron():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    F = np.array([(sx, sy, sz) for sx in (0, 1) for sy in (2, 3) for sz in (4, 5)], np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def _tetrahedron():
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float64)
    F = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def test_laplacian_of_regular_solids_and_euler():
    """Degrees 5 (icosahedron), 4 (octahedron), 3 (tetrahedron); rows sum to
    zero; symmetric; a closed genus-0 mesh has V - E + F = 2, E = 3F/2."""
    for (V, F), deg, ne in [(S.icosphere(0), 5, 30), (_octahedron(), 4, 12), (_tetrahedron(), 3, 6)]:
        nv = len(V)
        L = MU.laplacian(F, nv)
        assert len(MU.edges(F)) == ne
        np.testing.assert_array_equal(L.diagonal(), np.full(nv, deg))
        np.testing.assert_allclose(np.asarray(L.sum(axis=1)).ravel(), 0.0)
        assert abs(L - L.T).max() == 0
    V, F = S.icosphere(3)
    assert len(V) - len(MU.edges(F)) + len(F) == 2 and 2 * len(MU.edges(F)) == 3 * len(F)


def test_smooth_solve_keeps_constants_and_the_mean():
    """(I + lam L)^-1 fixes constant fields (L 1 = 0), keeps the mean of any
    field (1^T L = 0), is the identity at lam = 0 and shrinks the rest
    (eigenvalues 1 / (1 + lam mu) <= 1)."""
    V, F = S.icosphere(2)
    nv = len(V)
    rng = np.random.default_rng(81)
    c = np.array([0.3, -1.2, 2.0])
    np.testing.assert_allclose(MU.smooth_solve(F, nv, 7.0, np.tile(c, (nv, 1))), np.tile(c, (nv, 1)), rtol=1e-12)
    b = rng.normal(size=(nv, 3))
    x = MU.smooth_solve(F, nv, 7.0, b)
    np.testing.assert_allclose(x.mean(axis=0), b.mean(axis=0), rtol=1e-10, atol=1e-13)
    assert np.linalg.norm(x - x.mean(axis=0)) < np.linalg.norm(b - b.mean(axis=0))
    np.testing.assert_allclose(MU.smooth_solve(F, nv, 0.0, b), b, rtol=1e-14)


def test_adam_uniform_constant_gradient_closed_form():
    """With the same gradient every step the bias-corrected moments are g and
    max g^2, so every step is lr g / (max |g| + eps)."""
    rng = np.random.default_rng(82)
    g = rng.normal(size=(40, 3))
    st = None
    for _ in range(5):
        step, st = MU.adam_uniform(st, g, lr=0.01)
        np.testing.assert_allclose(step, 0.01 * g / (np.abs(g).max() + 1e-8), rtol=1e-12)


def test_large_steps_update_translates_under_a_constant_gradient():
    """A constant gradient c is a fixed point of the solve, so the update is
    the translation -lr c / (max |c| + eps) of every vertex."""
    V, F = S.icosphere(2)
    V = V.astype(np.float64)
    c = np.array([0.5, -2.0, 1.0])
    V1, st = MU.large_steps_update(F, V, np.tile(c, (len(V), 1)), None, lam=12.0, lr=0.01)
    np.testing.assert_allclose(V1, V - 0.01 * c / (2.0 + 1e-8), rtol=1e-10, atol=1e-12)


def test_edge_loss_closed_forms():
    """Unit vertex normals of a regular solid are radial: adjacent octahedron
    vertices are 90 degrees apart (each edge (1 - 0)^2 = 1), adjacent
    tetrahedron vertices have cos = -1/3 (each edge (4/3)^2 = 16/9); a flat
    patch has one normal (0)."""
    V, F = _octahedron()
    assert MU.edge_loss(V, F)[0] == pytest.approx(1.0, abs=1e-14)
    V, F = _tetrahedron()
    assert MU.edge_loss(V, F)[0] == pytest.approx(16.0 / 9.0, rel=1e-13)
    P = np.array([[x, y, 0.0] for y in range(4) for x in range(4)])
    F = np.array([[y * 4 + x, y * 4 + x + 1, (y + 1) * 4 + x] for y in range(3) for x in range(3)] +
                 [[y * 4 + x + 1, (y + 1) * 4 + x + 1, (y + 1) * 4 + x] for y in range(3) for x in range(3)])
    assert MU.edge_loss(P, F)[0] == pytest.approx(0.0, abs=1e-28)


def test_edge_loss_gradient_matches_central_differences():
    V, F = S.icosphere(1)
    rng = np.random.default_rng(83)
    V = V.astype(np.float64) * (1.0 + 0.1 * rng.uniform(size=(len(V), 1)))
    _, g = MU.edge_loss(V, F)
    eps = 1e-6
    fd = np.zeros_like(V)
    for idx in np.ndindex(V.shape):
        p, m = V.copy(), V.copy()
        p[idx] += eps
        m[idx] -= eps
        fd[idx] = (MU.edge_loss(p, F)[0] - MU.edge_loss(m, F)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_edges_ignore_repeated_vertices_and_faces():
    """A repeated face adds no edge and a face (a, a, b) adds only {a, b}."""
    F = np.array([[0, 1, 2], [0, 1, 2], [3, 3, 1]])
    np.testing.assert_array_equal(MU.edges(F), [[0, 1], [0, 2], [1, 2], [1, 3]])
