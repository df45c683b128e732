"""GB300 (sm_103a) recursive differentiable transparent-mesh ray tracer.

DiffTrans (arXiv 2603.00413), Sec. 3.3-3.4: camera rays traced through a
closed triangle mesh, split at every hit into Fresnel-weighted reflected and
Snell-refracted rays, attenuated inside by Beer-Lambert absorption, reading an
environment map where they escape; with the adjoint that returns image-loss
gradients for vertex positions, IoR and absorption.

This module is a thin ctypes binding of ``libdifftrans.so`` (C ABI in
``include/difftrans.h``): it marshals torch CUDA tensors into pointers and
sizes, and allocates the workspaces the library asks for.  Every step of the
computation runs in the library's kernels; there is no CPU path.  If the
library has not been built the calls raise instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import torch

__all__ = [
    "DiffTransError", "load_library", "vertex_normals", "vertex_normals_backward", "Bvh", "build_bvh",
    "refit_bvh", "Params", "render", "render_backward", "read_stats", "dump_segments", "closest_hit",
    "render_workspace_size", "backward_workspace_size", "Tape", "DiffTransRender", "render_differentiable",
    "l2_loss_grad", "profile_enable", "profile_read", "vertex_normals_noalloc", "BatchItem", "render_batch",
    "render_batch_backward", "batch_backward_workspace_size", "get_tuning", "set_tuning",
    "measure_l2_read_bandwidth",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdifftrans.so")

DT_OK = 0
DT_ERR_INVALID_ARG = 1
DT_ERR_CUDA = 2
DT_ERR_QUEUE_OVERFLOW = 3
DT_ERR_STACK_OVERFLOW = 4
DT_ERR_NOT_IMPLEMENTED = 5

SF_INSIDE, SF_TIR, SF_BACKFACING, SF_DISCARDED, SF_MISS = 4, 8, 16, 128, 512


class DiffTransError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"difftrans error {code}: {msg}")
        self.code = code


MAX_HASH_LEVELS = 16  # DT_MAX_HASH_LEVELS


class DtMedium(ctypes.Structure):
    _fields_ = [("d_mu", c_void_p), ("d_grad_mu", c_void_p), ("nx", c_int32), ("ny", c_int32), ("nz", c_int32),
                ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("step", ctypes.c_float),
                ("levels", c_int32), ("log2_table", c_int32), ("res", c_int32 * MAX_HASH_LEVELS)]


class DtScene(ctypes.Structure):
    _fields_ = [("d_V", c_void_p), ("d_F", c_void_p), ("nv", c_int32), ("nf", c_int32), ("d_bvh", c_void_p),
                ("d_N", c_void_p), ("d_ior", c_void_p), ("d_sigma", c_void_p), ("d_env", c_void_p),
                ("env_w", c_int32), ("env_h", c_int32), ("medium", ctypes.POINTER(DtMedium)),
                ("d_grad_env", c_void_p)]


class DtViews(ctypes.Structure):
    _fields_ = [("d_cams", c_void_p), ("n_views", c_int32), ("width", c_int32), ("height", c_int32)]


class DtParams(ctypes.Structure):
    _fields_ = [("max_depth", c_int32), ("spp", c_int32), ("jitter", c_int32), ("tape_mode", c_int32),
                ("seed", c_uint64), ("t_min", c_float), ("level_capacity", c_int32)]


class DtStats(ctypes.Structure):
    _fields_ = [("status", c_int32), ("n_levels", c_int32), ("segments", c_int64), ("seg_needed", c_int64),
                ("level_count", c_int64 * 32), ("level_start", c_int64 * 32), ("hits", c_int64),
                ("misses", c_int64), ("discarded", c_int64), ("backfacing", c_int64), ("tir", c_int64),
                ("nodes_visited", c_int64), ("tris_tested", c_int64), ("max_level", c_int64),
                ("level_needed", c_int64), ("medium_samples", c_int64)]

    def as_dict(self):
        n = self.n_levels
        return {
            "status": self.status, "n_levels": n, "segments": self.segments, "seg_needed": self.seg_needed,
            "level_count": list(self.level_count[:max(n, 1)]), "hits": self.hits, "misses": self.misses,
            "discarded": self.discarded, "backfacing": self.backfacing, "tir": self.tir,
            "nodes_visited": self.nodes_visited, "tris_tested": self.tris_tested, "max_level": self.max_level,
            "level_needed": self.level_needed, "medium_samples": self.medium_samples,
        }


class DtBatchEntry(ctypes.Structure):
    _fields_ = [("scene", DtScene), ("views", DtViews), ("params", DtParams), ("d_out", c_void_p),
                ("d_grad_out", c_void_p), ("d_grad_V", c_void_p), ("d_grad_ior", c_void_p),
                ("d_grad_sigma", c_void_p)]


class DtTuning(ctypes.Structure):
    _fields_ = [("trace_steps", c_int32), ("trace_refill", c_int32), ("trace_blocks_per_sm", c_int32),
                ("shade_blocks_per_sm", c_int32), ("bvh_width", c_int32), ("bvh_builder", c_int32),
                ("trace_order", c_int32), ("order_min_rays", c_int32)]


class DtKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", c_int64), ("total_ms", ctypes.c_double)]


# exported symbol -> (restype, argtypes)
_PROTOS = {
    "dt_last_error": (c_char_p, []),
    "dt_version": (c_char_p, []),
    "dt_vertex_normals_scratch_size": (c_int32, [c_int32, POINTER(c_size_t)]),
    "dt_vertex_normals": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "dt_vertex_normals_noalloc": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p]),
    "dt_vertex_normals_backward": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "dt_bvh_size": (c_int32, [c_int32, POINTER(c_size_t), POINTER(c_size_t)]),
    "dt_build_bvh": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "dt_refit_bvh": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "dt_render_workspace_size": (c_int32, [c_int64, POINTER(c_size_t)]),
    "dt_render_workspace_size_ex": (c_int32, [c_int64, c_int32, c_int64, POINTER(c_size_t)]),
    "dt_render": (c_int32, [POINTER(DtScene), POINTER(DtViews), POINTER(DtParams), c_void_p, c_void_p, c_size_t,
                            c_void_p]),
    "dt_read_stats": (c_int32, [c_void_p, c_size_t, POINTER(DtStats), c_void_p]),
    "dt_backward_workspace_size": (c_int32, [c_int64, c_int32, POINTER(c_size_t)]),
    "dt_render_backward": (c_int32, [POINTER(DtScene), POINTER(DtViews), POINTER(DtParams), c_void_p, c_size_t,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_int64,
                                     c_void_p]),
    "dt_dump_segments": (c_int32, [c_void_p, c_size_t, c_void_p, c_void_p, c_int64, c_void_p]),
    "dt_closest_hit": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_float, c_void_p,
                                 c_void_p, c_void_p]),
    "dt_render_batch": (c_int32, [POINTER(DtBatchEntry), c_int32, c_void_p, c_size_t, c_void_p]),
    "dt_batch_backward_workspace_size": (c_int32, [POINTER(DtBatchEntry), c_int32, c_int64, POINTER(c_size_t)]),
    "dt_render_batch_backward": (c_int32, [POINTER(DtBatchEntry), c_int32, c_void_p, c_size_t, c_void_p, c_size_t,
                                           c_int64, c_void_p]),
    "dt_l2_loss_grad": (c_int32, [c_void_p, c_void_p, c_int64, c_float, c_void_p, c_void_p, c_void_p]),
    "dt_paper_loss_grad": (c_int32, [c_void_p, c_void_p, c_int64, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "dt_topology_size": (c_int32, [c_int32, c_int32, POINTER(c_size_t)]),
    "dt_build_topology": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_size_t, c_void_p]),
    "dt_topology_info": (c_int32, [c_void_p, c_int32, c_int32, POINTER(c_int64), POINTER(c_int32),
                                   POINTER(c_void_p), POINTER(c_void_p), c_void_p]),
    "dt_smooth_scratch_size": (c_int32, [c_int32, c_int32, POINTER(c_size_t)]),
    "dt_smooth_solve": (c_int32, [c_void_p, c_int32, c_int32, c_float, c_void_p, c_void_p, c_int32, c_void_p, c_size_t,
                                  c_void_p]),
    "dt_large_steps_sizes": (c_int32, [c_int32, c_int32, POINTER(c_size_t), POINTER(c_size_t)]),
    "dt_large_steps_update": (c_int32, [c_void_p, c_int32, c_int32, c_float, c_float, c_float, c_float, c_float,
                                        c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "dt_edge_loss_grad": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dt_profile_enable": (c_int32, [c_int32]),
    "dt_get_tuning": (c_int32, [POINTER(DtTuning)]),
    "dt_set_tuning": (c_int32, [POINTER(DtTuning)]),
    "dt_measure_l2_read_bandwidth": (c_int32, [c_void_p, c_size_t, c_int32, POINTER(ctypes.c_double), c_void_p]),
    "dt_profile_read": (c_int32, [POINTER(DtKernelTime), c_int32, POINTER(c_int32)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdifftrans.so (built by ``paper_2603_00413_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2603_00413_gb300.build` "
                               "(there is no fallback implementation)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(code):
    if code != DT_OK:
        msg = load_library().dt_last_error().decode(errors="replace")
        raise DiffTransError(code, msg)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def _ptr(t):
    return c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, shape_tail=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} must end in shape {shape_tail}, got {tuple(t.shape)}")
    return t


def _aligned_empty(nbytes: int, device, align: int = 256):
    """A uint8 buffer whose data pointer is `align`-byte aligned (returns the
    owning tensor and the aligned view)."""
    raw = torch.empty(nbytes + align, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % align
    return raw, raw[off:off + nbytes]


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
_scratch_cache = {}


def _normals_scratch(nv, device):
    b = c_size_t()
    _check(load_library().dt_vertex_normals_scratch_size(nv, ctypes.byref(b)))
    key = (device, b.value)
    if key not in _scratch_cache:
        _scratch_cache.clear()
        _scratch_cache[key] = _aligned_empty(b.value, device)
    return _scratch_cache[key][1]


def vertex_normals(V, F, out=None, stream=None, scratch=None):
    """Eq. 13 vertex normals: (1/3) * sum of unit face normals per vertex
    (bit-reproducible: fixed-point accumulation in a scratch buffer)."""
    _need(V, torch.float32, (3,), "V")
    _need(F, torch.int32, (3,), "F")
    N = torch.empty_like(V) if out is None else out
    scratch = _normals_scratch(V.shape[0], V.device) if scratch is None else scratch
    _check(load_library().dt_vertex_normals(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(N), _ptr(scratch),
                                            _stream(stream)))
    return N


NOALLOC_MAX_VERTICES = 1 << 20
SEG_F = 15  # floats per segment of dump_segments


def vertex_normals_noalloc(V, F, out, stream=None):
    """Eq. 13 normals for callers that cannot allocate device memory: the
    scratch lives in a fixed 24 MiB array inside the library (at most 2^20
    vertices); `out` must be given.  Calls that overlap on the GPU share that
    array and race: keep them on one stream."""
    _need(V, torch.float32, (3,), "V")
    _need(F, torch.int32, (3,), "F")
    _need(out, torch.float32, (3,), "out")
    _check(load_library().dt_vertex_normals_noalloc(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(out),
                                                    _stream(stream)))
    return out


def vertex_normals_backward(V, F, dN, dV=None, stream=None):
    """dV += (dN/dV)^T dN for the Eq. 13 normals."""
    dV = torch.zeros_like(V) if dV is None else dV
    _check(load_library().dt_vertex_normals_backward(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(dN), _ptr(dV),
                                                     _stream(stream)))
    return dV


class Bvh:
    """An LBVH built by the library into a caller-owned device buffer."""

    def __init__(self, nf: int, device):
        bb, sb = c_size_t(), c_size_t()
        _check(load_library().dt_bvh_size(nf, ctypes.byref(bb), ctypes.byref(sb)))
        self.nf = nf
        self.bytes = bb.value
        self._raw, self.buf = _aligned_empty(bb.value, device)
        self._sraw, self.scratch = _aligned_empty(sb.value, device)

    def build(self, V, F, stream=None):
        _need(V, torch.float32, (3,), "V")
        _need(F, torch.int32, (3,), "F")
        _check(load_library().dt_build_bvh(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(self.buf),
                                           _ptr(self.scratch), _stream(stream)))
        return self

    def refit(self, V, F, stream=None):
        _check(load_library().dt_refit_bvh(_ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(self.buf),
                                           _ptr(self.scratch), _stream(stream)))
        return self


def build_bvh(V, F, stream=None) -> Bvh:
    return Bvh(F.shape[0], V.device).build(V, F, stream)


def refit_bvh(bvh: Bvh, V, F, stream=None) -> Bvh:
    return bvh.refit(V, F, stream)


def closest_hit(bvh: Bvh, o, d, src=None, t_min: float = 1e-5, stream=None):
    """Closest hit of arbitrary rays through the BVH: (tri int32 [n], tbb [n,3])."""
    _need(o, torch.float32, (3,), "o")
    _need(d, torch.float32, (3,), "d")
    n = o.shape[0]
    tri = torch.empty(n, dtype=torch.int32, device=o.device)
    tbb = torch.empty(n, 3, dtype=torch.float32, device=o.device)
    _check(load_library().dt_closest_hit(_ptr(bvh.buf), bvh.nf, _ptr(o), _ptr(d), _ptr(src), n, float(t_min),
                                         _ptr(tri), _ptr(tbb), _stream(stream)))
    return tri, tbb


# ---------------------------------------------------------------------------
# render / backward
# ---------------------------------------------------------------------------
class Params:
    """Render parameters.  checkpoint=True keeps only the per-depth ray
    queues on the tape and recovers the hits in the backward from the
    source triangle each spawned child carries
    (tape_mode 1); the hit ring then holds level_capacity records per level
    (0: chosen from the workspace, else twice the camera rays).
    moments=True (tape_mode 2) keeps the full tape plus, for the interior
    segments of a scene with an absorption grid or hash texture, the
    medium's optical depth and its derivatives (96 bytes per segment), so
    the backward does not read the medium's values again."""

    def __init__(self, max_depth: int, spp: int = 1, jitter: int = 0, seed: int = 0, t_min: float = 1e-5,
                 checkpoint: bool = False, level_capacity: int = 0, moments: bool = False):
        if checkpoint and moments:
            raise ValueError("a tape is either checkpointed or keeps the medium moments, not both")
        self.max_depth, self.spp, self.jitter, self.seed, self.t_min = max_depth, spp, jitter, seed, t_min
        self.checkpoint, self.level_capacity = bool(checkpoint), int(level_capacity)
        self.moments = bool(moments)

    def c(self, level_capacity: int = None):
        ring = self.level_capacity if level_capacity is None else level_capacity
        mode = 1 if self.checkpoint else (2 if self.moments else 0)
        return DtParams(self.max_depth, self.spp, self.jitter, mode, self.seed & (2 ** 64 - 1),
                        self.t_min, int(ring) if self.checkpoint else 0)


def render_workspace_size(seg_capacity: int, level_capacity: int = 0, moments: bool = False) -> int:
    """Bytes of a workspace for seg_capacity segments; level_capacity > 0
    sizes a checkpointed one (hit ring of that many records per level),
    moments=True one that keeps the medium moments (tape_mode 2)."""
    b = c_size_t()
    if level_capacity > 0:
        _check(load_library().dt_render_workspace_size_ex(int(seg_capacity), 1, int(level_capacity),
                                                          ctypes.byref(b)))
    elif moments:
        _check(load_library().dt_render_workspace_size_ex(int(seg_capacity), 2, 0, ctypes.byref(b)))
    else:
        _check(load_library().dt_render_workspace_size(int(seg_capacity), ctypes.byref(b)))
    return b.value


def backward_workspace_size(max_level: int, nv: int) -> int:
    b = c_size_t()
    _check(load_library().dt_backward_workspace_size(int(max_level), int(nv), ctypes.byref(b)))
    return b.value


class Workspace:
    """A caller-owned segment arena (the tape) for dt_render; level_capacity
    > 0 makes it a checkpointed one (hits of two levels only)."""

    def __init__(self, seg_capacity: int, device, level_capacity: int = 0, moments: bool = False):
        self.capacity = int(seg_capacity)
        self.level_capacity = int(min(level_capacity, self.capacity)) if level_capacity > 0 else 0
        self.moments = bool(moments) and not self.level_capacity
        self.bytes = render_workspace_size(self.capacity, self.level_capacity, self.moments)
        self._raw, self.buf = _aligned_empty(self.bytes, device)


class Medium:
    """Spatially varying absorption (Eq. 11 with mu_t(x) = sigma + G(x)): a
    grid of per-channel rates at the nodes of a lattice over the box [lo,
    hi], trilinear, positions clamped to the box; interior segments add the
    sum of G over steps of length `step` (the last one partial), each
    sampled at its midpoint.  mu: float32 device tensor [nz, ny, nx, 3] or
    [nz, ny, nx, 4] (stored with a 4th unused channel)."""

    def __init__(self, mu, lo, hi, step: float):
        if mu.dim() != 4 or mu.shape[3] not in (3, 4) or min(mu.shape[:3]) < 2:
            raise ValueError("mu must be [nz, ny, nx, 3 or 4] with at least 2 nodes per axis")
        if mu.shape[3] == 3:
            mu = torch.cat([mu, torch.zeros_like(mu[..., :1])], dim=3)
        self.mu = _need(mu.contiguous(), torch.float32, (4,), "mu")
        self.lo = tuple(float(x) for x in lo)
        self.hi = tuple(float(x) for x in hi)
        self.step = float(step)

    @property
    def shape(self):
        return tuple(self.mu.shape[:3])

    def struct(self, grad=None) -> DtMedium:
        m = DtMedium()
        m.d_mu = self.mu.data_ptr()
        m.d_grad_mu = grad.data_ptr() if grad is not None else None
        m.nz, m.ny, m.nx = self.mu.shape[0], self.mu.shape[1], self.mu.shape[2]
        for a in range(3):
            m.lo[a] = self.lo[a]
            m.hi[a] = self.hi[a]
        m.step = self.step
        return m


class HashTexture:
    """Spatially varying absorption given as a multi-resolution hash texture
    (Sec. 3.3's differentiable 3D texture, after Instant-NGP): L <= 16
    lattices over the box [lo, hi], level l with res[l] nodes per axis and
    its values in table[l] (T entries, T a power of two, 16 <= T <= 2^24):
    corner (i, j, k) at entry (k res + j) res + i when res^3 <= T, else at
    (i XOR 2654435761 j XOR 805459861 k) mod T.  G(x) is the sum of the
    levels' trilinear interpolations; steps along interior segments as for
    Medium.  table: float32 device tensor [L, T, 3] or [L, T, 4]; the
    gradient comes back as [L, T, 3]."""

    def __init__(self, table, res, lo, hi, step: float):
        res = [int(r) for r in res]
        if table.dim() != 3 or table.shape[2] not in (3, 4) or not 1 <= table.shape[0] <= MAX_HASH_LEVELS:
            raise ValueError(f"table must be [L, T, 3 or 4] with 1 <= L <= {MAX_HASH_LEVELS}")
        T = table.shape[1]
        if T < 16 or T > (1 << 24) or T & (T - 1):
            raise ValueError("the table size per level must be a power of two in 16..2^24")
        if len(res) != table.shape[0] or min(res) < 2 or max(res) > (1 << 20):
            raise ValueError("res needs one node count in 2..2^20 per level")
        if table.shape[2] == 3:
            table = torch.cat([table, torch.zeros_like(table[..., :1])], dim=2)
        self.mu = _need(table.contiguous(), torch.float32, (4,), "table")
        self.res = res
        self.lo = tuple(float(x) for x in lo)
        self.hi = tuple(float(x) for x in hi)
        self.step = float(step)

    def struct(self, grad=None) -> DtMedium:
        m = DtMedium()
        m.d_mu = self.mu.data_ptr()
        m.d_grad_mu = grad.data_ptr() if grad is not None else None
        for a in range(3):
            m.lo[a] = self.lo[a]
            m.hi[a] = self.hi[a]
        m.step = self.step
        m.levels = len(self.res)
        m.log2_table = self.mu.shape[1].bit_length() - 1
        for l, r in enumerate(self.res):
            m.res[l] = r
        return m


def _scene_struct(V, F, bvh, N, ior, sigma, env, medium_c=None, denv=None):
    _need(V, torch.float32, (3,), "V")
    _need(F, torch.int32, (3,), "F")
    _need(N, torch.float32, (3,), "N")
    _need(env, torch.float32, (3,), "env")
    _need(ior, torch.float32, None, "ior")
    _need(sigma, torch.float32, None, "sigma")
    if ior.numel() != 1 or sigma.numel() != 3:
        raise ValueError("ior needs 1 element and sigma 3")
    sc = DtScene(V.data_ptr(), F.data_ptr(), V.shape[0], F.shape[0], bvh.buf.data_ptr(), N.data_ptr(),
                 ior.data_ptr(), sigma.data_ptr(), env.data_ptr(), env.shape[1], env.shape[0])
    if medium_c is not None:
        sc.medium = ctypes.pointer(medium_c)
    if denv is not None:
        sc.d_grad_env = _need(denv, torch.float32, (3,), "d_grad_env").data_ptr()
    return sc


def _views_struct(cams, width, height):
    _need(cams, torch.float32, (10,), "cams")
    return DtViews(cams.data_ptr(), cams.shape[0], int(width), int(height))


def read_stats(ws: Workspace, stream=None) -> dict:
    st = DtStats()
    _check(load_library().dt_read_stats(_ptr(ws.buf), ws.bytes, ctypes.byref(st), _stream(stream)))
    return st.as_dict()


class Tape:
    """Everything dt_render_backward needs from a forward call (params_c:
    the dt_params the forward ran with)."""

    def __init__(self, ws, scene_args, cams, width, height, params, stats, params_c=None, medium=None):
        self.ws, self.scene_args, self.cams = ws, scene_args, cams
        self.width, self.height, self.params, self.stats = width, height, params, stats
        self.params_c = params_c if params_c is not None else params.c()
        self.medium = medium


def default_capacity(n_primary: int, max_depth: int) -> int:
    """First guess of the segment arena: 2D + 3 segments per primary ray is
    what a convex object needs; the arena grows on overflow."""
    return int(min(2 ** 31 - 1, max(n_primary * (2 * max_depth + 3), 1024)))


def _new_workspace(params: Params, n_primary: int, device, capacity: int = None, level_capacity: int = None):
    cap = default_capacity(n_primary, params.max_depth) if capacity is None else capacity
    if not params.checkpoint:
        return Workspace(cap, device, moments=params.moments)
    ring = level_capacity or params.level_capacity or 2 * n_primary
    return Workspace(cap, device, level_capacity=max(ring, 1))


def _grow_workspace(ws: Workspace, params: Params, stats: dict, device):
    """A larger workspace after an overflow of the arena or of a checkpointed
    level's hit ring."""
    cap = ws.capacity
    if stats["seg_needed"] > cap:
        cap = min(max(2 * cap, int(1.3 * stats["seg_needed"])), 2 ** 31 - 1)
    if not ws.level_capacity:
        return Workspace(cap, device, moments=ws.moments)
    ring = ws.level_capacity
    if stats["level_needed"] > ring:
        ring = int(1.25 * stats["level_needed"])
    return Workspace(max(cap, ring), device, level_capacity=ring)


def _effective_params(params: Params, ws: Workspace):
    if params.checkpoint and not ws.level_capacity:
        raise ValueError("a checkpointed render needs a workspace made with level_capacity > 0")
    if params.moments != ws.moments:
        raise ValueError("Params(moments=...) and the workspace's moments must agree")
    return params.c(ws.level_capacity if params.checkpoint else 0)


def render(V, F, bvh: Bvh, N, ior, sigma, env, cams, width: int, height: int, params: Params, ws: Workspace = None,
           out=None, stream=None, check: bool = True, medium=None):
    """Forward render (Sec. 3.4 steps 1-5) of cams.shape[0] views; medium:
    an absorption grid (Medium) or hash texture (HashTexture) added to sigma
    on interior segments.

    Returns (image [n_views, height, width, 3], Tape).  With check=True the
    device status is read back (one synchronisation) and an arena overflow is
    retried with a larger workspace."""
    lib = load_library()
    n_views = cams.shape[0]
    n0 = n_views * width * height * params.spp
    if ws is None:
        ws = _new_workspace(params, n0, V.device)
    if out is None:
        out = torch.empty(n_views, height, width, 3, dtype=torch.float32, device=V.device)
    mc = medium.struct() if medium is not None else None
    sc = _scene_struct(V, F, bvh, N, ior, sigma, env, mc)
    vw = _views_struct(cams, width, height)
    while True:
        pc = _effective_params(params, ws)
        _check(lib.dt_render(ctypes.byref(sc), ctypes.byref(vw), ctypes.byref(pc), _ptr(out), _ptr(ws.buf),
                             ws.bytes, _stream(stream)))
        if not check:
            return out, Tape(ws, (V, F, bvh, N, ior, sigma, env), cams, width, height, params, None, pc, medium)
        stats = read_stats(ws, stream)
        if stats["status"] == DT_ERR_QUEUE_OVERFLOW:
            ws = _grow_workspace(ws, params, stats, V.device)
            continue
        if stats["status"] != DT_OK:
            raise DiffTransError(stats["status"], "device-side error during render")
        return out, Tape(ws, (V, F, bvh, N, ior, sigma, env), cams, width, height, params, stats, pc, medium)


def render_backward(tape: Tape, grad_out, stream=None, bws=None, env_grad: bool = False):
    """Gradient of sum(grad_out * image) w.r.t. (V, ior, sigma) at the
    forward's fixed events.  Returns (dV [nv,3], dior [1], dsigma [3]),
    then dmu [nz, ny, nx, 3] when the render had an absorption grid (the
    table's [L, T, 3] for a hash texture), then denv [env_h, env_w, 3] when
    env_grad is set."""
    lib = load_library()
    V, F, bvh, N, ior, sigma, env = tape.scene_args
    stats = tape.stats if tape.stats is not None else read_stats(tape.ws, stream)
    if stats["status"] != DT_OK:
        raise DiffTransError(stats["status"], "the forward render did not finish cleanly")
    grad_out = _need(grad_out.contiguous(), torch.float32, (3,), "grad_out")
    max_level = max(1, stats["max_level"])
    nbytes = backward_workspace_size(max_level, V.shape[0])
    if bws is None or bws.numel() < nbytes:
        _, bws = _aligned_empty(nbytes, V.device)
    dV = torch.empty_like(V)
    dior = torch.empty(1, dtype=torch.float32, device=V.device)
    dsig = torch.empty(3, dtype=torch.float32, device=V.device)
    med = tape.medium
    dmu = torch.empty_like(med.mu) if med is not None else None
    mc = med.struct(dmu) if med is not None else None
    denv = torch.empty_like(env) if env_grad else None
    sc = _scene_struct(V, F, bvh, N, ior, sigma, env, mc, denv)
    vw = _views_struct(tape.cams, tape.width, tape.height)
    pc = tape.params_c
    _check(lib.dt_render_backward(ctypes.byref(sc), ctypes.byref(vw), ctypes.byref(pc), _ptr(tape.ws.buf),
                                  tape.ws.bytes, _ptr(grad_out), _ptr(dV), _ptr(dior), _ptr(dsig), _ptr(bws),
                                  bws.numel(), max_level, _stream(stream)))
    out = (dV, dior, dsig)
    if med is not None:
        out += (dmu[..., :3],)
    if env_grad:
        out += (denv,)
    return out


def dump_segments(tape: Tape, stream=None):
    """Every segment of the tape: (seg_i int32 [n,4] = (sample, heap node, tri,
    flags), seg_f float32 [n,15] = (t, b1, b2, origin, direction, throughput
    W, contribution W * E(d) of an escaped segment or 0))."""
    if tape.ws.level_capacity:
        raise ValueError("a checkpointed tape keeps no hit records to dump")
    if tape.ws.moments:
        raise ValueError("dump_segments reads tapes of tape_mode 0 only (this one keeps medium moments)")
    stats = tape.stats if tape.stats is not None else read_stats(tape.ws, stream)
    n = stats["segments"]
    dev = tape.ws.buf.device
    si = torch.empty(max(n, 1), 4, dtype=torch.int32, device=dev)
    sf = torch.empty(max(n, 1), SEG_F, dtype=torch.float32, device=dev)
    _check(load_library().dt_dump_segments(_ptr(tape.ws.buf), tape.ws.bytes, _ptr(si), _ptr(sf), n,
                                           _stream(stream)))
    return si[:n], sf[:n]


def l2_loss_grad(img, target, grad=None, loss=None, stream=None):
    """Mean-squared image loss and its gradient, in the library's kernel:
    loss = mean((img - target)^2), grad = 2 (img - target) / n."""
    _need(img, torch.float32, None, "img")
    _need(target, torch.float32, None, "target")
    n = img.numel()
    grad = torch.empty_like(img) if grad is None else grad
    loss = torch.empty(1, dtype=torch.float32, device=img.device) if loss is None else loss
    _check(load_library().dt_l2_loss_grad(_ptr(img), _ptr(target), n, 1.0 / max(n, 1), _ptr(grad), _ptr(loss),
                                          _stream(stream)))
    return grad, loss


def paper_loss_grad(img, target, lambda_color: float = 1.0, lambda_tone: float = 1.0, grad=None, loss=None,
                    stream=None):
    """The tracer stage's losses on the device (Eq. 14, GT-weighted L2, and
    Eq. 15, tone, per pixel and averaged): returns (d total / d img, loss
    [3] = (lambda_color L_color + lambda_tone L_tone, L_color, L_tone))."""
    _need(img, torch.float32, (3,), "img")
    _need(target, torch.float32, (3,), "target")
    if img.shape != target.shape:
        raise ValueError("img and target need the same shape")
    n = img.numel() // 3
    grad = torch.empty_like(img) if grad is None else grad
    loss = torch.empty(3, dtype=torch.float32, device=img.device) if loss is None else loss
    _check(load_library().dt_paper_loss_grad(_ptr(img), _ptr(target), n, float(lambda_color), float(lambda_tone),
                                             _ptr(grad), _ptr(loss), _stream(stream)))
    return grad, loss


# ---------------------------------------------------------------------------
# the step after the gradient (App. A)
# ---------------------------------------------------------------------------
class Topology:
    """The distinct neighbours of every vertex of a triangle mesh (CSR, on
    the device), for the large-steps update and L_edge."""

    def __init__(self, F, nv: int, stream=None):
        _need(F, torch.int32, (3,), "F")
        self.nv, self.nf = int(nv), F.shape[0]
        b = c_size_t()
        lib = load_library()
        _check(lib.dt_topology_size(self.nv, self.nf, ctypes.byref(b)))
        self.bytes = b.value
        self._raw, self.buf = _aligned_empty(self.bytes, F.device)
        _check(lib.dt_build_topology(_ptr(F), self.nf, self.nv, _ptr(self.buf), self.bytes, _stream(stream)))
        self._info = None

    def info(self, stream=None):
        """(distinct edges, largest neighbour count, row [nv + 1], col
        [2 edges]) -- synchronises once."""
        if self._info is None:
            ne, md = c_int64(), c_int32()
            rp, cp = c_void_p(), c_void_p()
            _check(load_library().dt_topology_info(_ptr(self.buf), self.nv, self.nf, ctypes.byref(ne),
                                                   ctypes.byref(md), ctypes.byref(rp), ctypes.byref(cp),
                                                   _stream(stream)))
            base = self.buf.data_ptr()
            row = self.buf[rp.value - base: rp.value - base + 4 * (self.nv + 1)].view(torch.int32)
            col = self.buf[cp.value - base: cp.value - base + 8 * ne.value].view(torch.int32)
            self._info = (ne.value, md.value, row, col)
        return self._info


def smooth_solve(topo: Topology, lam: float, b, x=None, iters: int = 100, stream=None):
    """x = (I + lam L)^-1 b (b [nv, 3]; x the start, overwritten) by
    preconditioned conjugate gradients on the device."""
    _need(b, torch.float32, (3,), "b")
    x = torch.zeros_like(b) if x is None else x
    s = c_size_t()
    lib = load_library()
    _check(lib.dt_smooth_scratch_size(topo.nv, int(iters), ctypes.byref(s)))
    _, scratch = _aligned_empty(s.value, b.device)
    _check(lib.dt_smooth_solve(_ptr(topo.buf), topo.nv, topo.nf, float(lam), _ptr(b), _ptr(x), int(iters),
                               _ptr(scratch), s.value, _stream(stream)))
    return x


class LargeStepsOptimizer:
    """The mesh update of the tracer stage: AdamUniform on u = (I + lam L) V
    with the gradient taken through the same matrix (Nicolet et al. 2021;
    learning rate 1e-3 in App. A).  step(dJ/dV) updates V in place."""

    def __init__(self, V, F, lam: float = 10.0, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8,
                 iters: int = 100, topo: Topology = None):
        _need(V, torch.float32, (3,), "V")
        self.V, self.F = V, F
        self.topo = topo if topo is not None else Topology(F, V.shape[0])
        self.lam, self.lr, self.betas, self.eps, self.iters = float(lam), float(lr), betas, float(eps), int(iters)
        st, sc = c_size_t(), c_size_t()
        _check(load_library().dt_large_steps_sizes(V.shape[0], self.iters, ctypes.byref(st), ctypes.byref(sc)))
        self._sraw, self.state = _aligned_empty(st.value, V.device)
        self.state.zero_()
        self._craw, self.scratch = _aligned_empty(sc.value, V.device)

    def step(self, grad, stream=None):
        _need(grad, torch.float32, (3,), "grad")
        _check(load_library().dt_large_steps_update(
            _ptr(self.topo.buf), self.topo.nv, self.topo.nf, self.lam, self.lr, float(self.betas[0]),
            float(self.betas[1]), self.eps, self.iters, _ptr(self.V), _ptr(grad.contiguous()), _ptr(self.state),
            _ptr(self.scratch), self.scratch.numel(), _stream(stream)))
        return self.V


def edge_loss_grad(V, F, topo: Topology = None, stream=None):
    """L_edge of App. A and its gradient with respect to the vertices
    (through the unit normals, Eq. 13 and the face cross products): returns
    (loss [1], dV [nv, 3])."""
    topo = topo if topo is not None else Topology(F, V.shape[0])
    N = vertex_normals(V, F, stream=stream)
    dN = torch.empty_like(N)
    loss = torch.empty(1, dtype=torch.float32, device=V.device)
    _check(load_library().dt_edge_loss_grad(_ptr(topo.buf), topo.nv, topo.nf, _ptr(N), _ptr(dN), _ptr(loss),
                                            _stream(stream)))
    return loss, vertex_normals_backward(V, F, dN, stream=stream)


def measure_l2_read_bandwidth(nbytes: int = 32 << 20, iters: int = 50, device=None, stream=None) -> float:
    """L2 read bandwidth (GB/s) of the current GPU, measured by the library."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    _, buf = _aligned_empty(nbytes, dev)
    buf.zero_()
    g = ctypes.c_double()
    _check(load_library().dt_measure_l2_read_bandwidth(_ptr(buf), nbytes, iters, ctypes.byref(g), _stream(stream)))
    return g.value


def get_tuning() -> dict:
    t = DtTuning()
    _check(load_library().dt_get_tuning(ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in DtTuning._fields_}


def set_tuning(**kw) -> dict:
    """Set launch/scheduling knobs (trace_steps, trace_refill,
    trace_blocks_per_sm, shade_blocks_per_sm, bvh_width, bvh_builder,
    trace_order, order_min_rays); returns the previous values."""
    old = get_tuning()
    new = dict(old)
    new.update(kw)
    t = DtTuning(*[int(new[f]) for f, _ in DtTuning._fields_])
    _check(load_library().dt_set_tuning(ctypes.byref(t)))
    return old


def profile_enable(on: bool = True):
    _check(load_library().dt_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    buf = (DtKernelTime * 64)()
    n = c_int32()
    _check(load_library().dt_profile_read(buf, 64, ctypes.byref(n)))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(min(n.value, 64))}


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------
class BatchItem:
    """One scene of a batched render: geometry, materials, environment, views
    and parameters, with its own output image."""

    def __init__(self, V, F, bvh: Bvh, N, ior, sigma, env, cams, width: int, height: int, params: Params,
                 medium=None):
        self.V, self.F, self.bvh, self.N = V, F, bvh, N
        self.ior, self.sigma, self.env, self.cams = ior, sigma, env, cams
        self.width, self.height, self.params = int(width), int(height), params
        self.medium = medium
        self.out = None

    @property
    def n_primary(self):
        return self.cams.shape[0] * self.width * self.height * self.params.spp

    def entry(self, out=None, grad_out=None, dV=None, dior=None, dsig=None, level_capacity: int = 0, dmu=None,
              denv=None):
        e = DtBatchEntry()
        # the medium struct must outlive the call: keep it on the item
        self._medium_c = self.medium.struct(dmu) if self.medium is not None else None
        e.scene = _scene_struct(self.V, self.F, self.bvh, self.N, self.ior, self.sigma, self.env, self._medium_c,
                                denv)
        e.views = _views_struct(self.cams, self.width, self.height)
        e.params = self.params.c(level_capacity)
        e.d_out = out.data_ptr() if out is not None else None
        e.d_grad_out = grad_out.data_ptr() if grad_out is not None else None
        e.d_grad_V = dV.data_ptr() if dV is not None else None
        e.d_grad_ior = dior.data_ptr() if dior is not None else None
        e.d_grad_sigma = dsig.data_ptr() if dsig is not None else None
        return e


class BatchTape:
    def __init__(self, ws, items, stats):
        self.ws, self.items, self.stats = ws, items, stats


def render_batch(items, ws: Workspace = None, outs=None, stream=None, check: bool = True):
    """Forward render of a batch of scenes in one set of launches.  Returns
    (list of images, BatchTape); with check=True the status is read back and
    an arena overflow retried."""
    lib = load_library()
    n = len(items)
    dev = items[0].V.device
    n0 = sum(it.n_primary for it in items)
    depth = max(it.params.max_depth for it in items)
    p0 = items[0].params
    if any(it.params.checkpoint != p0.checkpoint or it.params.moments != p0.moments for it in items):
        raise ValueError("all items of a batch share the tape mode (checkpoint, moments)")
    if ws is None:
        ws = _new_workspace(Params(depth, checkpoint=p0.checkpoint, level_capacity=p0.level_capacity,
                                   moments=p0.moments), n0, dev)
    if outs is None:
        outs = [torch.empty(it.cams.shape[0], it.height, it.width, 3, dtype=torch.float32, device=dev)
                for it in items]
    while True:
        if p0.checkpoint and not ws.level_capacity:
            raise ValueError("a checkpointed render needs a workspace made with level_capacity > 0")
        if p0.moments != ws.moments:
            raise ValueError("Params(moments=...) and the workspace's moments must agree")
        arr = (DtBatchEntry * n)(*[it.entry(out=o, level_capacity=ws.level_capacity) for it, o in zip(items, outs)])
        _check(lib.dt_render_batch(arr, n, _ptr(ws.buf), ws.bytes, _stream(stream)))
        if not check:
            return outs, BatchTape(ws, items, None)
        stats = read_stats(ws, stream)
        if stats["status"] == DT_ERR_QUEUE_OVERFLOW:
            ws = _grow_workspace(ws, p0, stats, dev)
            continue
        if stats["status"] != DT_OK:
            raise DiffTransError(stats["status"], "device-side error during render")
        return outs, BatchTape(ws, items, stats)


def batch_backward_workspace_size(items, max_level: int) -> int:
    arr = (DtBatchEntry * len(items))(*[it.entry(level_capacity=1) for it in items])
    b = c_size_t()
    _check(load_library().dt_batch_backward_workspace_size(arr, len(items), int(max_level), ctypes.byref(b)))
    return b.value


def render_batch_backward(tape: BatchTape, grads, bws=None, outs=None, stream=None, env_grad: bool = False):
    """Gradients of sum_i sum(grads[i] * image_i) for every scene of the
    batch: list of (dV, dior, dsigma), with dmu [nz, ny, nx, 3] appended for
    an item with an absorption grid ([L, T, 3] for a hash texture) and denv
    [env_h, env_w, 3] when env_grad is set."""
    lib = load_library()
    items = tape.items
    stats = tape.stats if tape.stats is not None else read_stats(tape.ws, stream)
    if stats["status"] != DT_OK:
        raise DiffTransError(stats["status"], "the forward render did not finish cleanly")
    max_level = max(1, stats["max_level"])
    nbytes = batch_backward_workspace_size(items, max_level)
    dev = items[0].V.device
    if bws is None or bws.numel() < nbytes:
        _, bws = _aligned_empty(nbytes, dev)
    if outs is None:
        outs = [(torch.empty_like(it.V), torch.empty(1, device=dev), torch.empty(3, device=dev)) for it in items]
    dmus = [torch.empty_like(it.medium.mu) if it.medium is not None else None for it in items]
    denvs = [torch.empty_like(it.env) if env_grad else None for it in items]
    grads = [_need(g.contiguous(), torch.float32, (3,), "grad") for g in grads]
    arr = (DtBatchEntry * len(items))(*[it.entry(grad_out=g, dV=o[0], dior=o[1], dsig=o[2],
                                                 level_capacity=tape.ws.level_capacity, dmu=m, denv=de)
                                        for it, g, o, m, de in zip(items, grads, outs, dmus, denvs)])
    _check(lib.dt_render_batch_backward(arr, len(items), _ptr(tape.ws.buf), tape.ws.bytes, _ptr(bws), bws.numel(),
                                        max_level, _stream(stream)))
    return [tuple(o) + ((m[..., :3],) if m is not None else ()) + ((de,) if de is not None else ())
            for o, m, de in zip(outs, dmus, denvs)]


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class DiffTransRender(torch.autograd.Function):
    """image = render(V, ior, sigma); backward through render_backward and the
    vertex-normal adjoint (both in the library)."""

    @staticmethod
    def forward(ctx, V, ior, sigma, F, env, cams, width, height, params, bvh):
        V = V.detach().contiguous()
        N = vertex_normals(V, F)
        if bvh is None:
            bvh = build_bvh(V, F)
        img, tape = render(V, F, bvh, N, ior.detach(), sigma.detach(), env, cams, width, height, params)
        ctx.tape = tape
        return img

    @staticmethod
    def backward(ctx, grad_img):
        dV, dior, dsig = render_backward(ctx.tape, grad_img.contiguous())
        ctx.tape = None
        return dV, dior, dsig, None, None, None, None, None, None, None


def render_differentiable(V, F, ior, sigma, env, cams, width, height, params: Params, bvh: Bvh = None):
    """Differentiable render: gradients flow to V, ior and sigma.  Builds the
    LBVH for V unless a BVH already built or refitted for V is given."""
    return DiffTransRender.apply(V, ior, sigma, F, env, cams, width, height, params, bvh)
