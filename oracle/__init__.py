"""FP64 brute-force oracle for the recursive transparent-mesh tracer.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The CUDA library never
imports, links or calls anything here, and nothing here touches the library.

The arithmetic lives in ``difftrans_oracle.cpp`` (plain C++, double precision,
OpenMP over pixels); this module compiles it with g++ on first use and wraps
its C entry points with ctypes.  Each wrapper names the part of the paper
(DiffTrans, arXiv 2603.00413) it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "difftrans_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liborc_difftrans.so")
_lock = threading.Lock()
_lib = None

# segment flag bits, same meaning as in difftrans_oracle.cpp
SEG_NEAR_EDGE = 1
SEG_NEAR_TIE = 2
SEG_INSIDE = 4
SEG_TIR = 8
SEG_BACKFACING = 16
SEG_NEAR_CRITICAL = 32
SEG_GRAZING = 64
SEG_DISCARDED = 128
SEG_NEAR_POLE = 256
SEG_MISS = 512
SEG_UNSTABLE = 1024
SEG_DEGENERATE = SEG_NEAR_EDGE | SEG_NEAR_TIE | SEG_NEAR_CRITICAL | SEG_GRAZING | SEG_NEAR_POLE | SEG_UNSTABLE

SEG_F = 15  # doubles per segment record (see render)
COUNTER_NAMES = ("segments", "hits", "misses", "discarded", "leaks", "backfacing", "tir", "degenerate")


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            # no fused multiply-add: the same FP64 results on x86 and Arm hosts, and
            # exactly zero cross products for parallel edges
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        U64 = ctypes.c_uint64
        I64 = ctypes.c_int64
        lib.orc_vertex_normals.argtypes = [P, I, P, I, P]
        lib.orc_closest_hit.argtypes = [P, I, P, I, P, P, P, I, D, P, P, P, P, P]
        lib.orc_interface.argtypes = [P, P, P, P, I, P, P, P, P, P]
        lib.orc_env_lookup.argtypes = [P, I, I, P, I, P]
        lib.orc_camera_rays.argtypes = [P, I, I, I, I, U64, I, P, P]
        lib.orc_pcg_hash.argtypes = [ctypes.c_uint32]
        lib.orc_pcg_hash.restype = ctypes.c_uint32
        M = ctypes.POINTER(_OrcMedium)
        lib.orc_render.argtypes = [P, I, P, I, D, P, P, I, I, P, I, I, I, I, I, U64, I, D, D,
                                   P, P, P, P, P, P, I64, P, P, M]
        lib.orc_render_rays.argtypes = [P, I, P, I, D, P, P, I, I, P, P, I, I, D, D,
                                        P, P, P, P, P, P, I64, P, P, M]
        lib.orc_render_jvp.argtypes = [P, I, P, I, D, P, P, I, I, P, I, I, I, I, I, U64, I, D,
                                       I, P, P, P, P, P, M, P]
        lib.orc_render_rays_jvp.argtypes = [P, I, P, I, D, P, P, I, I, P, P, I, I, D, I, P, P, P, P, P, M, P]
        lib.orc_trace_steps.argtypes = [P, I, P, I, D, P, P, I, I, P, P, P, P, I, I, D, P, P, M]
        lib.orc_medium_depth.argtypes = [M, P, P, P, I, P]
        lib.orc_field_eval.argtypes = [M, P, I, P]
        lib.orc_field_corners.argtypes = [M, P, I, P, P]
        _lib = lib
    return _lib


MAX_HASH_LEVELS = 16


class _OrcMedium(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("step", ctypes.c_double), ("levels", ctypes.c_int),
                ("log2_table", ctypes.c_int), ("res", ctypes.c_int * MAX_HASH_LEVELS)]


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _medium(medium):
    """(struct, keep-alive array) for a medium, or (None, None).  A dense
    grid is dict(mu [nz, ny, nx, 3], lo (3,), hi (3,), step); a hash texture
    is dict(table [L, T, 3] with T a power of two, res (L,) nodes per axis
    of each level, lo, hi, step)."""
    if medium is None:
        return None, None
    m = _OrcMedium()
    if "table" in medium:
        mu = _d(medium["table"])
        res = [int(r) for r in medium["res"]]
        L, T = mu.shape[0], mu.shape[1]
        assert mu.ndim == 3 and mu.shape[2] == 3 and 1 <= L <= MAX_HASH_LEVELS and len(res) == L
        assert T >= 2 and T & (T - 1) == 0 and min(res) >= 2
        m.levels, m.log2_table = L, T.bit_length() - 1
        for l, r in enumerate(res):
            m.res[l] = r
    else:
        mu = _d(medium["mu"])
        assert mu.ndim == 4 and mu.shape[3] == 3 and min(mu.shape[:3]) >= 2
        m.n[0], m.n[1], m.n[2] = mu.shape[2], mu.shape[1], mu.shape[0]
    m.mu = mu.ctypes.data_as(ctypes.c_void_p)
    for a in range(3):
        m.lo[a] = float(medium["lo"][a])
        m.hi[a] = float(medium["hi"][a])
    m.step = float(medium["step"])
    return m, mu


def _mp(m):
    return ctypes.byref(m) if m is not None else None


def medium_depth(medium, o, d, t) -> np.ndarray:
    """Optical depth of an absorption field over segments o + s d, s in
    [0, t] (Eq. 11 with the spatially varying rate): steps of length `step`
    from the start, the last one partial, each sampled at its midpoint with
    trilinear interpolation of the node values (positions clamped to the
    box); a hash texture sums its levels' interpolations (Sec. 3.3's 3D
    texture after Instant-NGP).  medium: a dense grid or a hash texture (see
    _medium).  Returns [n, 3]."""
    o, d = _d(o).reshape(-1, 3), _d(d).reshape(-1, 3)
    t = _d(t).reshape(-1)
    out = np.zeros_like(o)
    m, keep = _medium(medium)
    _load().orc_medium_depth(_mp(m), _p(o), _p(d), _p(t), o.shape[0], _p(out))
    del keep
    return out


def field_eval(medium, x) -> np.ndarray:
    """G at points x ([n, 3]) of a dense grid or hash texture: the value the
    optical-depth sum of Eq. 11 samples.  Returns [n, 3]."""
    x = _d(x).reshape(-1, 3)
    out = np.zeros_like(x)
    m, keep = _medium(medium)
    _load().orc_field_eval(_mp(m), _p(x), x.shape[0], _p(out))
    del keep
    return out


def field_corners(medium, x):
    """G at points x as a linear map of the values: (idx [n, K] int64, w
    [n, K]) with K = 8 corners per level (8 for a dense grid), idx the row of
    the flattened [entries, 3] values, so G(x_p) = sum_k w[p, k] *
    values[idx[p, k]]."""
    x = _d(x).reshape(-1, 3)
    levels = len(medium["res"]) if "table" in medium else 1
    K = 8 * levels
    idx = np.zeros((x.shape[0], K), np.int64)
    w = np.zeros((x.shape[0], K))
    m, keep = _medium(medium)
    _load().orc_field_corners(_mp(m), _p(x), x.shape[0], _p(idx), _p(w))
    del keep
    return idx, w


def _i(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def vertex_normals(V, F) -> np.ndarray:
    """Eq. 13: N_v = (1/3) * sum of unit normals of the faces around v."""
    V, F = _d(V), _i(F)
    N = np.zeros_like(V)
    _load().orc_vertex_normals(_p(V), V.shape[0], _p(F), F.shape[0], _p(N))
    return N


def closest_hit(V, F, o, d, src=None, t_min: float = 1e-5):
    """Brute-force closest hit over all triangles (Sec. 3.4 step 2)."""
    V, F, o, d = _d(V), _i(F), _d(o).reshape(-1, 3), _d(d).reshape(-1, 3)
    n = o.shape[0]
    s = _i(src) if src is not None else None
    tri = np.zeros(n, np.int32)
    t, b1, b2 = np.zeros(n), np.zeros(n), np.zeros(n)
    fl = np.zeros(n, np.int32)
    _load().orc_closest_hit(_p(V), V.shape[0], _p(F), F.shape[0], _p(o), _p(d), _p(s), n, t_min,
                            _p(tri), _p(t), _p(b1), _p(b2), _p(fl))
    return tri, t, b1, b2, fl


def interface(d, n, eta1, eta2):
    """Sec. 3.3: reflection (Eq. 3), refraction (Eqs. 4-6), TIR, Fresnel
    (Eqs. 7-8) at one interface.  d: incoming direction, n: shading normal on
    the incoming side."""
    d, n = _d(d).reshape(-1, 3), _d(n).reshape(-1, 3)
    m = d.shape[0]
    e1 = _d(np.broadcast_to(eta1, (m,)))
    e2 = _d(np.broadcast_to(eta2, (m,)))
    wr, wt = np.zeros((m, 3)), np.zeros((m, 3))
    R, T = np.zeros(m), np.zeros(m)
    tir = np.zeros(m, np.int32)
    _load().orc_interface(_p(d), _p(n), _p(e1), _p(e2), m, _p(wr), _p(wt), _p(R), _p(T), _p(tir))
    return wr, wt, R, T, tir.astype(bool)


def env_lookup(env, dirs) -> np.ndarray:
    """Bilinear equirectangular lookup (Sec. 3.4 step 3 with an environment map)."""
    env = _d(env)
    H, W = env.shape[0], env.shape[1]
    dirs = _d(dirs).reshape(-1, 3)
    out = np.zeros_like(dirs)
    _load().orc_env_lookup(_p(env), W, H, _p(dirs), dirs.shape[0], _p(out))
    return out


def camera_rays(cam, spp: int = 1, jitter: int = 0, seed: int = 0, view: int = 0):
    """Pinhole camera rays of one view, ray index (py*W + px)*spp + s."""
    c = _d(cam.as_array())
    n = cam.width * cam.height * spp
    o, d = np.zeros((n, 3)), np.zeros((n, 3))
    _load().orc_camera_rays(_p(c), cam.width, cam.height, spp, jitter, seed, view, _p(o), _p(d))
    return o, d


def pcg_hash(v: int) -> int:
    return int(_load().orc_pcg_hash(ctypes.c_uint32(v & 0xFFFFFFFF)))


def _common(V, F, ior, sigma, env, cam):
    return _d(V), _i(F), float(ior), _d(sigma).reshape(3), _d(env), _d(cam.as_array())


def render(V, F, ior, sigma, env, cam, max_depth: int, spp: int = 1, jitter: int = 0, seed: int = 0,
           view: int = 0, t_min: float = 1e-5, segments: bool = False, probe: float = 0.0, medium=None) -> dict:
    """FP64 render of one view: the recursive ray tree of Sec. 3.4 steps 1-5.

    Returns dict(img [H,W,3], discard [H,W,3], pix_flags [H,W], pix_sig [H,W],
    counters {...}) and, with segments=True, seg_i [n,4] = (ray, heap node,
    tri, flags) and seg_f [n,15] = (t, b1, b2, origin xyz, direction xyz,
    throughput W rgb, contribution W * E(d) rgb of an escaped segment, 0 for
    a hit); W is the product of the A R or A T factors of Sec. 3.4 steps 4-5
    over the segment's ancestors, so the sample's radiance is the sum of the
    contributions.
    discard is the path weight lost to the depth limit or to a backfacing
    shading normal.  probe > 0 re-traces every primary ray tilted by probe
    radians four ways and flags pixels whose path events change
    (SEG_UNSTABLE in pix_flags).  medium: an absorption grid (see
    medium_depth) added to sigma on interior segments."""
    V, F, ior, sigma, env, c = _common(V, F, ior, sigma, env, cam)
    m, keep = _medium(medium)
    H, W = cam.height, cam.width
    img = np.zeros((H * W, 3))
    disc = np.zeros((H * W, 3))
    pf = np.zeros(H * W, np.int32)
    sig = np.zeros(H * W, np.uint64)
    cnt = np.zeros(8, np.int64)
    nseg = np.zeros(1, np.int64)
    lib = _load()
    args = (_p(V), V.shape[0], _p(F), F.shape[0], ior, _p(sigma), _p(env), env.shape[1], env.shape[0],
            _p(c), W, H, int(max_depth), int(spp), int(jitter), int(seed), int(view), float(t_min), float(probe),
            _p(img), _p(disc), _p(pf), _p(sig))
    seg_i, seg_f = _run_with_segments(lib.orc_render, args, segments, nseg, cnt, m)
    del keep
    out = dict(img=img.reshape(H, W, 3), discard=disc.reshape(H, W, 3), pix_flags=pf.reshape(H, W),
               pix_sig=sig.reshape(H, W), counters=dict(zip(COUNTER_NAMES, cnt.tolist())))
    if segments:
        out["seg_i"], out["seg_f"] = seg_i, seg_f
    return out


def _run_with_segments(fn, args, segments, nseg, cnt, m=None):
    if not segments:
        fn(*args, None, None, 0, None, _p(cnt), _mp(m))
        return None, None
    fn(*args, None, None, 0, _p(nseg), _p(cnt), _mp(m))
    n = int(nseg[0])
    seg_i = np.zeros((max(n, 1), 4), np.int32)
    seg_f = np.zeros((max(n, 1), SEG_F))
    fn(*args, _p(seg_i), _p(seg_f), n, _p(nseg), _p(cnt), _mp(m))
    return seg_i[:n], seg_f[:n]


def render_rays(V, F, ior, sigma, env, o, d, max_depth: int, t_min: float = 1e-5,
                segments: bool = False, probe: float = 0.0, medium=None) -> dict:
    """The same FP64 ray tree for arbitrary primary rays (o, d: [n,3], d
    unit), one sample each.  Outputs as render() with pixels = rays."""
    V, F = _d(V), _i(F)
    sigma, env = _d(sigma).reshape(3), _d(env)
    o, d = _d(o).reshape(-1, 3), _d(d).reshape(-1, 3)
    n = o.shape[0]
    img = np.zeros((n, 3))
    disc = np.zeros((n, 3))
    pf = np.zeros(n, np.int32)
    sig = np.zeros(n, np.uint64)
    cnt = np.zeros(8, np.int64)
    nseg = np.zeros(1, np.int64)
    lib = _load()
    args = (_p(V), V.shape[0], _p(F), F.shape[0], float(ior), _p(sigma), _p(env), env.shape[1], env.shape[0],
            _p(o), _p(d), n, int(max_depth), float(t_min), float(probe), _p(img), _p(disc), _p(pf), _p(sig))
    m, keep = _medium(medium)
    seg_i, seg_f = _run_with_segments(lib.orc_render_rays, args, segments, nseg, cnt, m)
    del keep
    out = dict(img=img, discard=disc, pix_flags=pf, pix_sig=sig, counters=dict(zip(COUNTER_NAMES, cnt.tolist())))
    if segments:
        out["seg_i"], out["seg_f"] = seg_i, seg_f
    return out


def trace_steps(V, F, ior, sigma, env, o, d, src, k, max_depth: int, t_min: float = 1e-5, medium=None):
    """One step of the FP64 tree (Sec. 3.4 steps 1-5) from each of n given
    segments: origin o [n,3], unit direction d [n,3], the triangle it leaves
    src [n] (-1: none) and its depth index k [n].  Returns (seg_i [n,3,4],
    seg_f [n,3,SEG_F]): the records of the segment (node 1) and of its
    reflected (node 2) and refracted (node 3) child, as render() writes them
    with the segment's throughput set to 1; node 0 marks a child that does
    not exist.  A child's own hit is not shaded (its flags say discarded)."""
    V, F = _d(V), _i(F)
    sigma, env = _d(sigma).reshape(3), _d(env)
    o, d = _d(o).reshape(-1, 3), _d(d).reshape(-1, 3)
    n = o.shape[0]
    src, k = _i(np.broadcast_to(src, (n,))), _i(np.broadcast_to(k, (n,)))
    seg_i = np.zeros((max(n, 1), 3, 4), np.int32)
    seg_f = np.zeros((max(n, 1), 3, SEG_F))
    m, keep = _medium(medium)
    _load().orc_trace_steps(_p(V), V.shape[0], _p(F), F.shape[0], float(ior), _p(sigma), _p(env), env.shape[1],
                            env.shape[0], _p(o), _p(d), _p(src), _p(k), n, int(max_depth), float(t_min), _p(seg_i),
                            _p(seg_f), _mp(m))
    del keep
    return seg_i[:n], seg_f[:n]


def render_jvp(V, F, ior, sigma, env, cam, max_depth: int, tV=None, tior=None, tsigma=None,
               spp: int = 1, jitter: int = 0, seed: int = 0, view: int = 0, t_min: float = 1e-5,
               medium=None, tmu=None):
    """Forward-mode derivative of the FP64 render along ntan directions at
    fixed events.  tV: [ntan, nv, 3], tior: [ntan], tsigma: [ntan, 3], tmu:
    [ntan, nz, ny, nx, 3] (tangents of the absorption grid's node values;
    [ntan, L, T, 3] for a hash texture's table entries).
    Returns (img [H,W,3], dimg [ntan,H,W,3])."""
    V, F, ior, sigma, env, c = _common(V, F, ior, sigma, env, cam)
    m, keep = _medium(medium)
    tmu = _d(tmu) if tmu is not None else None
    nt = None
    for a in (tV, tior, tsigma, tmu):
        if a is not None:
            nt = np.asarray(a).shape[0]
    assert nt is not None and nt > 0
    tV = _d(tV) if tV is not None else None
    tior = _d(tior) if tior is not None else None
    tsigma = _d(tsigma) if tsigma is not None else None
    H, W = cam.height, cam.width
    img = np.zeros((H * W, 3))
    dimg = np.zeros((nt, H * W, 3))
    _load().orc_render_jvp(_p(V), V.shape[0], _p(F), F.shape[0], ior, _p(sigma), _p(env), env.shape[1],
                           env.shape[0], _p(c), W, H, int(max_depth), int(spp), int(jitter), int(seed),
                           int(view), float(t_min), nt, _p(tV), _p(tior), _p(tsigma), _p(img), _p(dimg),
                           _mp(m), _p(tmu))
    del keep
    return img.reshape(H, W, 3), dimg.reshape(nt, H, W, 3)


def render_rays_jvp(V, F, ior, sigma, env, o, d, max_depth: int, tV=None, tior=None, tsigma=None,
                    t_min: float = 1e-5, medium=None, tmu=None):
    """Forward-mode derivative of the FP64 tree of arbitrary primary rays
    (tangents as render_jvp).  Returns (radiance [n,3], d radiance
    [ntan,n,3])."""
    V, F = _d(V), _i(F)
    sigma, env = _d(sigma).reshape(3), _d(env)
    o, d = _d(o).reshape(-1, 3), _d(d).reshape(-1, 3)
    n = o.shape[0]
    m, keep = _medium(medium)
    tmu = _d(tmu) if tmu is not None else None
    nt = None
    for a in (tV, tior, tsigma, tmu):
        if a is not None:
            nt = np.asarray(a).shape[0]
    assert nt is not None and nt > 0
    tV = _d(tV) if tV is not None else None
    tior = _d(tior) if tior is not None else None
    tsigma = _d(tsigma) if tsigma is not None else None
    img = np.zeros((n, 3))
    dimg = np.zeros((nt, n, 3))
    _load().orc_render_rays_jvp(_p(V), V.shape[0], _p(F), F.shape[0], float(ior), _p(sigma), _p(env), env.shape[1],
                                env.shape[0], _p(o), _p(d), n, int(max_depth), float(t_min), nt, _p(tV), _p(tior),
                                _p(tsigma), _p(img), _p(dimg), _mp(m), _p(tmu))
    del keep
    return img, dimg


def support_vertices(F, tris):
    """Vertices whose positions can move the radiance of paths that hit the
    given triangles: the triangles' own vertices and, through the Eq. 13
    vertex normals, every vertex of a face that touches one of them."""
    F = np.asarray(F, dtype=np.int64)
    tris = np.unique(np.asarray(tris, dtype=np.int64))
    tris = tris[tris >= 0]
    core = np.unique(F[tris].reshape(-1))
    touching = np.isin(F, core).any(axis=1)
    return np.unique(np.concatenate([core, F[touching].reshape(-1)]))


def rays_grad(V, F, ior, sigma, env, o, d, max_depth: int, g, t_min: float = 1e-5, chunk: int = 256):
    """Gradient of J = sum(g * radiance(rays)) w.r.t. (V, ior, sigma) by
    forward mode over every parameter that can influence these rays (the
    support of their hit triangles); all other vertex gradients are 0.
    Returns (dV [nv,3], dior, dsigma [3], segments traced in the forward)."""
    V = _d(V)
    nv = V.shape[0]
    g = _d(g).reshape(-1, 3)
    fw = render_rays(V, F, ior, sigma, env, o, d, max_depth, t_min, segments=True)
    verts = support_vertices(F, fw["seg_i"][:, 2])
    tior = np.array([1.0, 0, 0, 0])
    tsig = np.zeros((4, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    _, dimg = render_rays_jvp(V, F, ior, sigma, env, o, d, max_depth, None, tior, tsig, t_min)
    J = np.einsum("knc,nc->k", dimg, g)
    coords = [(int(v), a) for v in verts for a in range(3)]
    dV = np.zeros((nv, 3))
    for s in range(0, len(coords), chunk):
        part = coords[s:s + chunk]
        tV = np.zeros((len(part), nv, 3))
        for j, (v, a) in enumerate(part):
            tV[j, v, a] = 1.0
        _, dd = render_rays_jvp(V, F, ior, sigma, env, o, d, max_depth, tV, None, None, t_min)
        Jv = np.einsum("knc,nc->k", dd, g)
        for j, (v, a) in enumerate(part):
            dV[v, a] = Jv[j]
    return dV, float(J[0]), J[1:4], int(fw["counters"]["segments"])


def grad_full(V, F, ior, sigma, env, cam, max_depth: int, g, vert_subset=None, chunk: int = 64, **kw):
    """Gradient of J = sum(g * I) w.r.t. (V, ior, sigma) by forward mode over
    every parameter (one tangent per coordinate).  vert_subset limits the
    vertex coordinates probed (others reported as 0).  Slow; small cases only.
    Returns (dV [nv,3], dior, dsigma [3])."""
    V = _d(V)
    nv = V.shape[0]
    g = _d(g)
    verts = np.arange(nv) if vert_subset is None else np.asarray(vert_subset)
    coords = [(int(v), a) for v in verts for a in range(3)]
    dV = np.zeros((nv, 3))
    # ior and sigma first
    tior = np.array([1.0, 0, 0, 0])
    tsig = np.zeros((4, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    _, dimg = render_jvp(V, F, ior, sigma, env, cam, max_depth, None, tior, tsig, **kw)
    J = np.einsum("khwc,hwc->k", dimg, g)
    dior, dsig = J[0], J[1:4]
    for s in range(0, len(coords), chunk):
        part = coords[s:s + chunk]
        tV = np.zeros((len(part), nv, 3))
        for j, (v, a) in enumerate(part):
            tV[j, v, a] = 1.0
        _, dimg = render_jvp(V, F, ior, sigma, env, cam, max_depth, tV, None, None, **kw)
        J = np.einsum("khwc,hwc->k", dimg, g)
        for j, (v, a) in enumerate(part):
            dV[v, a] = J[j]
    return dV, float(dior), dsig


def paper_losses(img, target, lambda_color: float = 1.0, lambda_tone: float = 1.0):
    """The training losses of the tracer stage, in FP64, with their gradient
    with respect to the rendered image (an array [..., 3] of pixel colours
    c_hat; target: the ground-truth colours c of the same shape).

    Eq. 14 (GT-weighted L2): L_color = (1/|B|) sum_i ||(c_hat_i - c_i) * c_i||^2
    over the |B| pixels, the product channel-wise.
    Eq. 15 (tone): L_tone = (1 - c_hat . c / (||c_hat|| ||c||))^2 - var(c),
    read per pixel (var = the population variance of the pixel's three
    ground-truth channels) and averaged over the pixels like Eq. 14; a pixel
    whose rendered or true colour is zero has no defined cosine and counts it
    as 0 (its term 1 - var(c), no gradient).
    Returns (total = lambda_color L_color + lambda_tone L_tone, L_color,
    L_tone, dTotal/dc_hat)."""
    ch = np.asarray(img, np.float64).reshape(-1, 3)
    c = np.asarray(target, np.float64).reshape(-1, 3)
    P = ch.shape[0]
    r = (ch - c) * c
    l_color = float((r * r).sum() / P)
    g_color = 2.0 * r * c / P
    nh = np.linalg.norm(ch, axis=1)
    nc = np.linalg.norm(c, axis=1)
    ok = (nh > 0) & (nc > 0)
    s = np.zeros(P)
    s[ok] = (ch[ok] * c[ok]).sum(axis=1) / (nh[ok] * nc[ok])
    var = c.var(axis=1)
    l_tone = float(((1.0 - s) ** 2 - var).sum() / P)
    ds = np.zeros_like(ch)
    ds[ok] = c[ok] / (nh[ok] * nc[ok])[:, None] - s[ok, None] * ch[ok] / (nh[ok] ** 2)[:, None]
    g_tone = (-2.0 * (1.0 - s))[:, None] * ds / P
    total = lambda_color * l_color + lambda_tone * l_tone
    grad = (lambda_color * g_color + lambda_tone * g_tone).reshape(np.shape(img))
    return total, l_color, l_tone, grad


def mat_smooth_loss(medium, v, xi):
    """L_mat-smooth of Sec. 3.4 (Eq. 16): (1/N) sum_i |mu_t(v_i) - mu_t(v_i +
    xi_i)| over N points v_i with perturbations xi_i (both drawn by the
    caller), |.| read as the sum of the three channels' absolute values;
    sigma cancels, so only the field G counts.  Returns (loss, dL/d(values))
    with the gradient in the shape of the medium's values ([nz, ny, nx, 3]
    or [L, T, 3]); a channel whose difference is exactly 0 contributes no
    gradient (the subgradient 0)."""
    v = _d(v).reshape(-1, 3)
    xi = _d(xi).reshape(-1, 3)
    N = v.shape[0]
    values = _d(medium["table"] if "table" in medium else medium["mu"])
    flat = values.reshape(-1, 3)
    ia, wa = field_corners(medium, v)
    ib, wb = field_corners(medium, v + xi)
    D = (wa[..., None] * flat[ia]).sum(axis=1) - (wb[..., None] * flat[ib]).sum(axis=1)
    loss = float(np.abs(D).sum() / max(N, 1))
    s = np.sign(D) / max(N, 1)
    g = np.zeros_like(flat)
    for c in range(3):
        np.add.at(g[:, c], ia.ravel(), (wa * s[:, c:c + 1]).ravel())
        np.add.at(g[:, c], ib.ravel(), -(wb * s[:, c:c + 1]).ravel())
    return loss, g.reshape(values.shape)
