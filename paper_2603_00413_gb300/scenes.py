"""Seeded synthetic inputs for the recursive transparent-mesh tracer.

This module makes the scenes the tracer runs on: closed, outward-oriented
triangle meshes (icosphere, iso-surfaces of signed-distance fields, a
grid-tessellated box), equirectangular environment maps, pinhole cameras and
request streams.  It holds none of the tracer's own arithmetic -- no ray
generation, intersection, vertex normals, shading or absorption -- so the
CUDA path and the FP64 oracle both take its outputs as plain inputs.

Every floating-point array it returns is rounded to float32 once; the oracle
widens those exact float32 values to float64, so both sides start from
bit-identical data.

The paper's datasets (synthetic NEMTO-style scenes and real captures, Sec. 4.1
and Table "dataset") are not available; these generators stand in for them
with the shapes the paper gives: ~100 views of one object on a sphere around
it, infinitely distant environment maps, IoRs in the range of Table "ior".
"""
from __future__ import annotations

import dataclasses
import itertools
import math
import os

import numpy as np

F32 = np.float32


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    """Pinhole look-at camera; all values are float32-representable."""
    eye: tuple
    at: tuple
    up: tuple
    fov_y_deg: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """[eye(3), at(3), up(3), fov_y_deg] as float32 (10 values)."""
        return np.array(list(self.eye) + list(self.at) + list(self.up) + [self.fov_y_deg], dtype=F32)


def _f32t(v):
    return tuple(float(F32(x)) for x in v)


def camera(eye, at=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_y_deg=45.0, width=64, height=64) -> Camera:
    return Camera(_f32t(eye), _f32t(at), _f32t(up), float(F32(fov_y_deg)), int(width), int(height))


def fibonacci_views(n: int, distance: float = 3.0, width: int = 512, height: int = 512,
                    fov_y_deg: float = 45.0) -> list:
    """n cameras on a Fibonacci sphere of the given radius, looking at the origin."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(n):
        y = 1.0 - 2.0 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - y * y))
        ph = golden * i
        eye = (distance * r * math.cos(ph), distance * y, distance * r * math.sin(ph))
        cams.append(camera(eye, (0, 0, 0), (0, 1, 0), fov_y_deg, width, height))
    return cams


def random_view(rng: np.random.Generator, distance: float, width: int, height: int,
                fov_y_deg: float = 45.0) -> Camera:
    """A camera at a uniformly random point of a sphere, looking at the origin."""
    while True:
        v = rng.normal(size=3)
        n = np.linalg.norm(v)
        if n > 1e-6 and abs(v[1] / n) < 0.995:
            break
    eye = distance * v / n
    return camera(eye, (0, 0, 0), (0, 1, 0), fov_y_deg, width, height)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def _orient_outward_convex(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Flip faces of a star-shaped (about the origin) mesh to point outward."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def icosphere(subdiv: int, radius: float = 1.0):
    """Icosahedron split `subdiv` times (each triangle into 4, midpoints pushed
    onto the sphere).  V = 10*4^s + 2, F = 20*4^s.  Returns float32 V, int32 F."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    base = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            base += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    P = np.array(base)
    # faces: vertex triples whose pairwise distances are all the edge length 2
    d = np.linalg.norm(P[:, None, :] - P[None, :, :], axis=-1)
    adj = np.abs(d - 2.0) < 1e-9
    faces = [t for t in itertools.combinations(range(12), 3)
             if adj[t[0], t[1]] and adj[t[1], t[2]] and adj[t[0], t[2]]]
    assert len(faces) == 20
    V = P / np.linalg.norm(P, axis=1, keepdims=True)
    F = np.array(faces, dtype=np.int64)
    for _ in range(subdiv):
        mid = {}
        verts = list(V)
        newF = []

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                m = (verts[i] + verts[j]) / 2.0
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        V = np.array(verts)
        F = np.array(newF, dtype=np.int64)
    F = _orient_outward_convex(V, F)
    return (V * radius).astype(F32), F.astype(np.int32)


def box_grid(n: int, half_extent=(1.0, 1.0, 1.0)):
    """Closed axis-aligned box whose six faces are each an n x n grid of squares
    (two triangles each), oriented outward.  Every vertex strictly inside a face
    touches only coplanar triangles."""
    hx, hy, hz = half_extent
    verts = {}
    vlist = []
    faces = []

    def vid(p):
        key = tuple(round(x, 12) for x in p)
        if key not in verts:
            verts[key] = len(vlist)
            vlist.append(p)
        return verts[key]

    lin = np.linspace(-1.0, 1.0, n + 1)
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    quad = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0.0, 0.0, 0.0]
                        p[axis] = sgn
                        p[u_ax] = lin[i + di]
                        p[v_ax] = lin[j + dj]
                        quad.append(vid(tuple(p)))
                    faces.append((quad[0], quad[1], quad[2]))
                    faces.append((quad[0], quad[2], quad[3]))
    V = np.array(vlist) * np.array([hx, hy, hz])
    F = np.array(faces, dtype=np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, (a + b + c) / 3.0) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V.astype(F32), F.astype(np.int32)


# Freudenthal (Kuhn) split of the unit cube into six tetrahedra along the main
# diagonal; neighbouring cubes split shared faces along the same diagonal, so
# the tetrahedralisation is conforming and the extracted surface is closed.
_CORNER = {(dx, dy, dz): (dx << 2) | (dy << 1) | dz for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)}
_TETS = []
for _perm in itertools.permutations(range(3)):
    _p = [0, 0, 0]
    _path = [_CORNER[tuple(_p)]]
    for _ax in _perm:
        _p[_ax] = 1
        _path.append(_CORNER[tuple(_p)])
    _TETS.append(_path)
_TETS = np.array(_TETS, dtype=np.int64)  # [6, 4] corner ids


def marching_tetrahedra(field: np.ndarray, lo: float, hi: float, clamp: float = 0.02):
    """Zero iso-surface of a sampled scalar field (negative = inside).

    field: [n, n, n] values at grid points lo + i*(hi-lo)/(n-1).  Each grid cube
    is cut into six tetrahedra; every tetrahedron with a sign change emits one
    triangle (1 or 3 corners inside) or two (2 inside).  Surface vertices sit on
    grid/tetrahedron edges at the linearly interpolated zero, the interpolation
    parameter clamped to [clamp, 1-clamp] so no triangle collapses; vertices on
    a shared edge are welded.  Faces are oriented from inside to outside.
    The field must be positive on the grid boundary so the surface is closed.
    Stands in for marching cubes: no ambiguous cases and no case table.
    """
    f = np.asarray(field, dtype=np.float64)
    n = f.shape[0]
    assert f.shape == (n, n, n)
    # keep every grid value away from exactly zero
    tiny = 1e-9 * max(1.0, float(np.abs(f).max()))
    f = np.where(np.abs(f) < tiny, tiny, f)
    if not ((f[0] > 0).all() and (f[-1] > 0).all() and (f[:, 0] > 0).all() and (f[:, -1] > 0).all()
            and (f[:, :, 0] > 0).all() and (f[:, :, -1] > 0).all()):
        raise ValueError("field must be positive on the grid boundary")
    h = (hi - lo) / (n - 1)
    # active cubes: sign change among the 8 corners
    m = n - 1
    cmin = np.full((m, m, m), np.inf)
    cmax = np.full((m, m, m), -np.inf)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                s = f[dx:dx + m, dy:dy + m, dz:dz + m]
                cmin = np.minimum(cmin, s)
                cmax = np.maximum(cmax, s)
    ci, cj, ck = np.nonzero((cmin < 0) & (cmax > 0))
    ci, cj, ck = ci.astype(np.int64), cj.astype(np.int64), ck.astype(np.int64)
    corner_gid = np.empty((ci.size, 8), dtype=np.int64)
    for (dx, dy, dz), c in _CORNER.items():
        corner_gid[:, c] = ((ci + dx) * n + (cj + dy)) * n + (ck + dz)
    tg = corner_gid[:, _TETS].reshape(-1, 4)  # [ntet, 4] grid ids
    fflat = f.reshape(-1)
    tv = fflat[tg]
    inside = tv < 0
    cnt = inside.sum(axis=1)
    tri_edges = []  # list of [k, 3, 2] arrays of (grid id a, grid id b) per triangle vertex
    tri_in = []     # [k, 3] reference position inside
    tri_out = []

    def emit(sel, edges, ins, outs):
        if not sel.any():
            return
        g = tg[sel]
        e = np.stack([np.stack([g[:, a], g[:, b]], axis=-1) for (a, b) in edges], axis=1)
        tri_edges.append(e)
        tri_in.append(np.stack([g[:, i] for i in ins], axis=1))
        tri_out.append(np.stack([g[:, o] for o in outs], axis=1))

    for pattern in range(1, 15):
        bits = [(pattern >> q) & 1 for q in range(4)]
        sel = (cnt == sum(bits))
        for q in range(4):
            sel &= inside[:, q] == bool(bits[q])
        if not sel.any():
            continue
        ins = [q for q in range(4) if bits[q]]
        outs = [q for q in range(4) if not bits[q]]
        if len(ins) == 1 or len(ins) == 3:
            lone = ins[0] if len(ins) == 1 else outs[0]
            others = [q for q in range(4) if q != lone]
            emit(sel, [(lone, others[0]), (lone, others[1]), (lone, others[2])], ins, outs)
        else:
            a, b = ins
            c, d = outs
            quad = [(a, c), (a, d), (b, d), (b, c)]
            emit(sel, [quad[0], quad[1], quad[2]], ins, outs)
            emit(sel, [quad[0], quad[2], quad[3]], ins, outs)
    E = np.concatenate(tri_edges, axis=0)  # [T, 3, 2]
    Gin = [x for x in tri_in]
    Gout = [x for x in tri_out]
    # edge key -> welded vertex
    ea = np.minimum(E[..., 0], E[..., 1])
    eb = np.maximum(E[..., 0], E[..., 1])
    key = ea * (n ** 3) + eb
    ukey, inv = np.unique(key.reshape(-1), return_inverse=True)
    ua = ukey // (n ** 3)
    ub = ukey % (n ** 3)
    fa, fb = fflat[ua], fflat[ub]
    t = np.clip(fa / (fa - fb), clamp, 1.0 - clamp)

    def gpos(g):
        k = g % n
        j = (g // n) % n
        i = g // (n * n)
        return lo + h * np.stack([i, j, k], axis=-1).astype(np.float64)

    pa, pb = gpos(ua), gpos(ub)
    V = pa + t[:, None] * (pb - pa)
    F = inv.reshape(-1, 3).astype(np.int64)
    # orientation: normal must point from the inside corners to the outside ones
    cin = np.concatenate([gpos(x).mean(axis=1) for x in Gin], axis=0)
    cout = np.concatenate([gpos(x).mean(axis=1) for x in Gout], axis=0)
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", nrm, cout - cin) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def check_closed_mesh(V: np.ndarray, F: np.ndarray) -> dict:
    """Structural checks: every edge in exactly two faces with opposite
    directions (closed, consistently oriented 2-manifold), positive signed
    volume (outward), no zero-area face.  Returns stats; raises on failure."""
    F = np.asarray(F, dtype=np.int64)
    nv = int(V.shape[0])
    d = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
    dk = d[:, 0] * nv + d[:, 1]
    if np.unique(dk).size != dk.size:
        raise ValueError("a directed edge appears twice (inconsistent orientation or non-manifold)")
    rk = d[:, 1] * nv + d[:, 0]
    if not np.isin(rk, dk).all():
        raise ValueError("an edge has no opposite half-edge (open mesh)")
    Vd = np.asarray(V, dtype=np.float64)
    a, b, c = Vd[F[:, 0]], Vd[F[:, 1]], Vd[F[:, 2]]
    vol = float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)
    area2 = np.linalg.norm(np.cross(b - a, c - a), axis=1)
    if vol <= 0:
        raise ValueError("signed volume is not positive (faces point inward)")
    if area2.min() <= 0:
        raise ValueError("zero-area face")
    used = np.zeros(nv, dtype=bool)
    used[F.reshape(-1)] = True
    euler = nv - d.shape[0] // 2 + F.shape[0]
    return {"nv": nv, "nf": int(F.shape[0]), "volume": vol, "genus": (2 - euler) // 2,
            "min_area2": float(area2.min()), "all_vertices_used": bool(used.all())}


def normalize_unit_sphere(V: np.ndarray) -> np.ndarray:
    """Centre the bounding box at the origin and scale so max |v| = 1."""
    V = np.asarray(V, dtype=np.float64)
    c = (V.min(axis=0) + V.max(axis=0)) / 2.0
    V = V - c
    return V / np.linalg.norm(V, axis=1).max()


def _finish_mesh(V, F):
    V32 = normalize_unit_sphere(V).astype(F32)
    F32i = np.asarray(F, dtype=np.int32)
    check_closed_mesh(V32, F32i)
    return V32, F32i


def _grid(lo, hi, n):
    x = np.linspace(lo, hi, n)
    return np.meshgrid(x, x, x, indexing="ij")


def _sdf_torus(X, Y, Z, c, R, r, rot=None):
    P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1)
    if rot is not None:
        P = P @ rot  # rows of rot are the torus frame axes
    q = np.sqrt(P[..., 0] ** 2 + P[..., 1] ** 2) - R
    return np.sqrt(q * q + P[..., 2] ** 2) - r


def _sdf_ellipsoid(X, Y, Z, c, radii, rot):
    P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ rot
    q = np.linalg.norm(P / np.asarray(radii), axis=-1)
    return (q - 1.0) * float(np.min(radii))


def _smin_poly(a, b, k):
    h = np.clip(0.5 + 0.5 * (b - a) / k, 0.0, 1.0)
    return b * (1.0 - h) + a * h - k * h * (1.0 - h)


def two_tori_mesh(grid: int = 72, R: float = 0.5, r: float = 0.2, sep: float = 0.45, k: float = 0.1):
    """Smooth union of two overlapping tori in the xy plane (genus 2), extracted
    on grid^3 points over [-1.2, 1.2]^3 and normalised to the unit sphere."""
    X, Y, Z = _grid(-1.2, 1.2, grid)
    a = _sdf_torus(X, Y, Z, (-sep, 0.0, 0.0), R, r)
    b = _sdf_torus(X, Y, Z, (sep, 0.0, 0.0), R, r)
    V, F = marching_tetrahedra(_smin_poly(a, b, k), -1.2, 1.2)
    return _finish_mesh(V, F)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def blob_prims(rng: np.random.Generator) -> list:
    """Parameters of a random SDF: 1-6 ellipsoids or tori with random axes,
    radii and centres in [-0.5, 0.5]^3 (plain data, picklable)."""
    prims = []
    for _ in range(int(rng.integers(1, 7))):
        c = rng.uniform(-0.5, 0.5, size=3)
        rot = _random_rotation(rng)
        if rng.uniform() < 0.5:
            prims.append(("e", c, rng.uniform(0.15, 0.5, size=3), rot))
        else:
            R = rng.uniform(0.2, 0.45)
            prims.append(("t", c, (R, rng.uniform(0.06, 0.45 * R)), rot))
    return prims


def random_blob_field(rng: np.random.Generator):
    """A random SDF: the union (min) of blob_prims(rng).  Returns a callable
    on grids."""
    return blob_field(blob_prims(rng))


def blob_field(prims):
    def field(X, Y, Z):
        out = None
        for kind, c, prm, rot in prims:
            if kind == "e":
                s = _sdf_ellipsoid(X, Y, Z, c, prm, rot)
            else:
                s = _sdf_torus(X, Y, Z, c, prm[0], prm[1], rot)
            out = s if out is None else np.minimum(out, s)
        return out
    return field


@dataclasses.dataclass
class BatchSpec:
    """One scene of the batching workload, as plain data."""
    index: int
    prims: list
    faces: int
    side: int
    depth: int
    ior: float
    sigma: np.ndarray
    env_seed: int
    cam_seed: int


def batch_specs(n: int = 64, seed: int = 2) -> list:
    """n scenes: faces log-uniform in [2k, 200k], square images with side
    log-uniform in [128, 800], depth uniform in 4..12, IoR ~ U[1.3, 1.7],
    per-channel absorption ~ U[0, 2], a 256x128 SH environment each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(BatchSpec(
            index=i, prims=blob_prims(rng),
            faces=int(round(math.exp(rng.uniform(math.log(2000), math.log(200000))))),
            side=int(round(math.exp(rng.uniform(math.log(128), math.log(800))))),
            depth=int(rng.integers(4, 13)), ior=float(F32(rng.uniform(1.3, 1.7))),
            sigma=rng.uniform(0.0, 2.0, size=3).astype(F32), env_seed=int(rng.integers(0, 2 ** 31)),
            cam_seed=int(rng.integers(0, 2 ** 31))))
    return out


def build_batch_scene(spec: BatchSpec) -> Scene:
    """The scene of one BatchSpec (top-level, so a process pool can run it)."""
    V, F = mesh_from_field(blob_field(spec.prims), spec.faces)
    env = sh_env_map(256, 128, spec.env_seed)
    cam = random_view(np.random.default_rng(spec.cam_seed), 3.0, spec.side, spec.side)
    return Scene(V, F, spec.ior, spec.sigma, env, [cam], spec.depth, 1, 0, spec.index)


def batch_scenes(n: int = 64, seed: int = 2, workers: int = None) -> list:
    """The batching workload (see batch_specs), built in parallel processes
    (spawned, so this is safe after CUDA has been initialised)."""
    specs = batch_specs(n, seed)
    workers = workers or min(len(specs), os.cpu_count() or 1)
    if workers <= 1:
        return [build_batch_scene(s) for s in specs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(build_batch_scene, specs, chunksize=1)


def serve_specs(n: int = 32, seed: int = 4) -> list:
    """The serving workload's resident meshes: n random blobs as in
    batch_specs, with faces log-uniform in [5k, 500k]; IoR ~ U[1.3, 1.7],
    absorption ~ U[0, 2], a 256x128 SH environment each (the requests pick
    their own view, size and depth)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(BatchSpec(
            index=i, prims=blob_prims(rng),
            faces=int(round(math.exp(rng.uniform(math.log(5000), math.log(500000))))),
            side=256, depth=8, ior=float(F32(rng.uniform(1.3, 1.7))),
            sigma=rng.uniform(0.0, 2.0, size=3).astype(F32), env_seed=int(rng.integers(0, 2 ** 31)),
            cam_seed=int(rng.integers(0, 2 ** 31))))
    return out


def serve_scenes(n: int = 32, seed: int = 4, workers: int = None) -> list:
    """The serving workload's meshes (serve_specs), built in spawned processes."""
    specs = serve_specs(n, seed)
    workers = workers or min(len(specs), os.cpu_count() or 1)
    if workers <= 1:
        return [build_batch_scene(s) for s in specs]
    import multiprocessing as mp
    # the largest meshes first, so they do not finish last on one worker
    order = sorted(range(len(specs)), key=lambda i: -specs[i].faces)
    with mp.get_context("spawn").Pool(workers) as pool:
        built = pool.map(build_batch_scene, [specs[i] for i in order], chunksize=1)
    out = [None] * len(specs)
    for i, sc in zip(order, built):
        out[i] = sc
    return out


def mesh_from_field(field, target_faces: int, lo: float = -1.2, hi: float = 1.2,
                    max_grid: int = 640):
    """Extract a field's iso-surface at the grid resolution that gives about
    `target_faces` triangles (face count grows as grid^2)."""
    n = 48
    for _ in range(3):
        X, Y, Z = _grid(lo, hi, n)
        V, F = marching_tetrahedra(field(X, Y, Z), lo, hi)
        ratio = target_faces / max(1, F.shape[0])
        if 0.9 < ratio < 1.1:
            break
        n = int(min(max_grid, max(16, round(n * math.sqrt(ratio)))))
    return _finish_mesh(V, F)


def _value_noise_3d(rng, X, Y, Z, freq):
    """Lattice value noise: random values on an integer lattice of spacing
    1/freq, blended with the quintic smoothstep."""
    size = int(math.ceil(freq * 3.0)) + 4
    lat = rng.uniform(-1.0, 1.0, size=(size, size, size))
    out = np.zeros_like(X)
    P = [(A + 1.5) * freq for A in (X, Y, Z)]
    I = [np.floor(p).astype(np.int64) for p in P]
    T = [p - i for p, i in zip(P, I)]
    S = [t * t * t * (t * (t * 6 - 15) + 10) for t in T]
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = (S[0] if dx else 1 - S[0]) * (S[1] if dy else 1 - S[1]) * (S[2] if dz else 1 - S[2])
                out += w * lat[I[0] + dx, I[1] + dy, I[2] + dz]
    return out


def noisy_sphere_mesh(grid: int, seed: int = 3, amplitude: float = 0.1, octaves: int = 3):
    """Sphere SDF (r = 1) plus `octaves` of value noise (lacunarity 2, gain 0.5)
    of the given amplitude, over [-1.3, 1.3]^3."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _grid(-1.3, 1.3, grid)
    f = np.sqrt(X * X + Y * Y + Z * Z) - 1.0
    amp, freq = amplitude, 2.0
    for _ in range(octaves):
        f = f + amp * _value_noise_3d(rng, X, Y, Z, freq)
        amp *= 0.5
        freq *= 2.0
    V, F = marching_tetrahedra(f, -1.3, 1.3)
    return _finish_mesh(V, F)


# --------------------------------------------------------------------------
# environment maps
# --------------------------------------------------------------------------
def _real_sh_basis(lmax: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonics Y_lm, l = 0..lmax, m = -l..l,
    evaluated in FP64 at polar angle theta (from +y) and azimuth phi.
    Returns [(lmax+1)^2, *theta.shape]."""
    x = np.cos(theta)
    out = []
    # associated Legendre P_l^m(x) by the standard three-term recurrences
    P = {}
    P[(0, 0)] = np.ones_like(x)
    somx2 = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    for m in range(1, lmax + 1):
        P[(m, m)] = -(2 * m - 1) * somx2 * P[(m - 1, m - 1)]
    for m in range(0, lmax):
        P[(m + 1, m)] = (2 * m + 1) * x * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(K * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2.0) * K * P[(l, am)] * np.cos(am * phi))
            else:
                out.append(math.sqrt(2.0) * K * P[(l, am)] * np.sin(am * phi))
    return np.stack(out, axis=0)


def texel_directions(width: int, height: int):
    """Unit directions of equirectangular texel centres (row i = polar angle
    (i+0.5)/H*pi from +y, column j = azimuth (j+0.5)/W*2pi from +x toward +z)."""
    th = (np.arange(height) + 0.5) / height * math.pi
    ph = (np.arange(width) + 0.5) / width * 2.0 * math.pi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    return TH, PH


def sh_env_map(width: int, height: int, seed: int, lmax: int = 4) -> np.ndarray:
    """Smooth random environment: real SH up to degree lmax with N(0,1)
    coefficients per channel from the seed, evaluated at texel centres in
    FP64, then softplus.  Returns float32 [height, width, 3]."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=((lmax + 1) ** 2, 3))
    TH, PH = texel_directions(width, height)
    Y = _real_sh_basis(lmax, TH, PH)  # [K, H, W]
    val = np.einsum("khw,kc->hwc", Y, coef)
    return np.logaddexp(0.0, val).astype(F32)


def constant_env(width: int, height: int, rgb=(1.0, 1.0, 1.0)) -> np.ndarray:
    return np.broadcast_to(np.asarray(rgb, dtype=F32), (height, width, 3)).copy()


# --------------------------------------------------------------------------
# absorption grids (a spatially varying absorption rate inside the object)
# --------------------------------------------------------------------------
def grid_nodes(n, lo, hi):
    """Node coordinates (X, Y, Z), each [nz, ny, nx], of a grid with n =
    (nx, ny, nz) nodes spanning the box [lo, hi]."""
    ax = [np.linspace(lo[a], hi[a], n[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def linear_absorption_grid(n, lo, hi, a, b, step: float) -> dict:
    """Node values of the per-channel field a_c + b_c . x (a: [3], b: [3, 3]
    with b[c] the gradient of channel c) on an (nx, ny, nz) grid over
    [lo, hi].  float64 node values; dict(mu [nz, ny, nx, 3], lo, hi, step)."""
    X, Y, Z = grid_nodes(n, lo, hi)
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    mu = np.stack([a[c] + b[c, 0] * X + b[c, 1] * Y + b[c, 2] * Z for c in range(3)], axis=-1)
    return dict(mu=mu, lo=tuple(map(float, lo)), hi=tuple(map(float, hi)), step=float(step))


def random_absorption_grid(n, lo, hi, seed: int, scale: float = 1.0, step: float = None) -> dict:
    """Smooth non-negative random absorption rates on an (nx, ny, nz) grid
    over [lo, hi]: value noise of two octaves per channel from the seed,
    softplus, times scale.  float32 node values; step defaults to half the
    smallest cell."""
    rng = np.random.default_rng(seed)
    X, Y, Z = grid_nodes(n, lo, hi)
    mu = np.zeros(X.shape + (3,))
    for c in range(3):
        v = _value_noise_3d(rng, X, Y, Z, 2.0) + 0.5 * _value_noise_3d(rng, X, Y, Z, 4.0)
        mu[..., c] = np.logaddexp(0.0, 2.0 * v - 0.5)
    cell = min((hi[a] - lo[a]) / (n[a] - 1) for a in range(3))
    return dict(mu=(scale * mu).astype(F32), lo=tuple(map(float, lo)), hi=tuple(map(float, hi)),
                step=float(F32(0.5 * cell if step is None else step)))


def hash_texture_resolutions(levels: int, n_min: int, n_max: int) -> list:
    """Nodes per axis of the levels of a multi-resolution hash texture,
    growing geometrically from n_min to n_max (Instant-NGP's level scale:
    factor b = exp((ln n_max - ln n_min) / (L - 1)), n_l = floor(n_min b^l))."""
    if levels == 1:
        return [int(n_min)]
    b = math.exp((math.log(n_max) - math.log(n_min)) / (levels - 1))
    return [int(math.floor(n_min * b ** l + 1e-6)) for l in range(levels)]


def random_hash_texture(levels: int, log2_table: int, n_min: int, n_max: int, lo, hi, seed: int,
                        scale: float = 1.0, step: float = None) -> dict:
    """A multi-resolution hash texture of per-channel absorption rates over
    [lo, hi]: table [levels, 2^log2_table, 3] of rates drawn uniformly from
    [0, 2 scale / levels) (so G, the sum of the levels, averages `scale`),
    float32; res from hash_texture_resolutions; step defaults to half the
    finest cell."""
    rng = np.random.default_rng(seed)
    res = hash_texture_resolutions(levels, n_min, n_max)
    table = rng.uniform(0.0, 2.0 * scale / levels, size=(levels, 1 << log2_table, 3)).astype(F32)
    cell = min((hi[a] - lo[a]) / (res[-1] - 1) for a in range(3))
    return dict(table=table, res=res, lo=tuple(map(float, lo)), hi=tuple(map(float, hi)),
                step=float(F32(0.5 * cell if step is None else step)))


# --------------------------------------------------------------------------
# the benchmark workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    V: np.ndarray          # float32 [nv, 3]
    F: np.ndarray          # int32 [nf, 3]
    ior: float
    sigma: np.ndarray      # float32 [3]
    env: np.ndarray        # float32 [H, W, 3]
    cams: list             # [Camera]
    max_depth: int
    spp: int = 1
    jitter: int = 0
    seed: int = 0


def glass_icosphere_scene(width=64, height=64, max_depth=4, seed=0, subdiv=3) -> Scene:
    """One glass icosphere (subdivision 3: 642 vertices, 1280 triangles,
    radius 1), IoR 1.5, no absorption, camera at distance 3 on +z, 64x64,
    1 sample at pixel centres, depth 4, 64x32 SH environment."""
    V, F = icosphere(subdiv, 1.0)
    env = sh_env_map(64, 32, seed)
    cam = camera((0.0, 0.0, 3.0), (0, 0, 0), (0, 1, 0), 45.0, width, height)
    return Scene(V, F, float(F32(1.5)), np.zeros(3, F32), env, [cam], max_depth, 1, 0, seed)


def genus2_scene(n_views=100, width=512, height=512, max_depth=8, seed=1, grid=72,
                 perturb=0.005):
    """Two-tori genus-2 mesh (about 50k triangles), IoR ~ U[1.3, 1.7], per
    channel absorption ~ U[0, 2], Fibonacci views at distance 3, 512x512,
    depth 8.  Returns (scene, perturbed vertices for the target render)."""
    rng = np.random.default_rng(seed)
    V, F = two_tori_mesh(grid)
    ior = float(F32(rng.uniform(1.3, 1.7)))
    sigma = rng.uniform(0.0, 2.0, size=3).astype(F32)
    env = sh_env_map(64, 32, seed)
    cams = fibonacci_views(n_views, 3.0, width, height)
    Vt = (V.astype(np.float64) + rng.normal(0.0, perturb, size=V.shape)).astype(F32)
    return Scene(V, F, ior, sigma, env, cams, max_depth, 1, 0, seed), Vt
