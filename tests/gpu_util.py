"""Shared helpers of the GPU tests: move a seeded scene to the device, run the
library through the Python binding, run the oracle on the same inputs, and
compare.  (Test harness only: it calls both sides, neither side calls it.)"""
import numpy as np
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S

# tolerances of the parity bar: FP32 against FP64 along paths of up to
# eight interactions (radiance), and the adjoint's FP32 accumulation (gradients)
RAD_RTOL = 1e-4
RAD_ATOL = 1e-6
GRAD_RTOL = 1e-3
# tilt (radians) of the oracle's stability probe: pixels whose path events
# change under it are the edge-degenerate ones excluded from parity
PROBE = 1e-6


def dev():
    return torch.device("cuda:0")


class GpuScene:
    def __init__(self, V, F, ior, sigma, env, cams, width, height, max_depth, spp=1, jitter=0, seed=0,
                 t_min=1e-5):
        d = dev()
        self.Vn = np.asarray(V, np.float32)
        self.Fn = np.asarray(F, np.int32)
        self.envn = np.asarray(env, np.float32)
        self.iorf = float(np.float32(ior))
        self.sigman = np.asarray(sigma, np.float32).reshape(3)
        self.cam_list = list(cams)
        self.V = torch.from_numpy(self.Vn).to(d)
        self.F = torch.from_numpy(self.Fn).to(d)
        self.ior = torch.tensor([self.iorf], dtype=torch.float32, device=d)
        self.sigma = torch.from_numpy(self.sigman).to(d)
        self.env = torch.from_numpy(self.envn).to(d)
        self.cams = torch.from_numpy(np.stack([c.as_array() for c in cams])).to(d)
        self.width, self.height = width, height
        self.params = dt.Params(max_depth, spp, jitter, seed, t_min)
        self.N = dt.vertex_normals(self.V, self.F)
        self.bvh = dt.build_bvh(self.V, self.F)

    @classmethod
    def from_scene(cls, sc: S.Scene, views=None, width=None, height=None, **kw):
        cams = sc.cams if views is None else [sc.cams[i] for i in views]
        w = width or cams[0].width
        h = height or cams[0].height
        cams = [S.camera(c.eye, c.at, c.up, c.fov_y_deg, w, h) for c in cams]
        return cls(sc.V, sc.F, sc.ior, sc.sigma, sc.env, cams, w, h, kw.pop("max_depth", sc.max_depth),
                   kw.pop("spp", sc.spp), kw.pop("jitter", sc.jitter), kw.pop("seed", sc.seed), **kw)

    def render(self, **kw):
        return dt.render(self.V, self.F, self.bvh, self.N, self.ior, self.sigma, self.env, self.cams, self.width,
                         self.height, self.params, **kw)

    def oracle(self, view=0, segments=False, probe=PROBE):
        p = self.params
        return O.render(self.Vn, self.Fn, self.iorf, self.sigman, self.envn, self.cam_list[view], p.max_depth,
                        p.spp, p.jitter, p.seed, view, p.t_min, segments=segments, probe=probe)


def degenerate_pixels(orc):
    return (orc["pix_flags"] & O.SEG_DEGENERATE) != 0


def assert_radiance_parity(img_gpu, orc, exclude=None):
    """Per pixel and channel |gpu - oracle| <= RAD_RTOL |oracle| + RAD_ATOL on
    pixels whose oracle path has no degenerate event."""
    g = img_gpu.detach().cpu().numpy().astype(np.float64)
    o = orc["img"]
    bad = degenerate_pixels(orc)
    if exclude is not None:
        bad = bad | exclude
    ok = ~bad
    err = np.abs(g - o)
    tol = RAD_RTOL * np.abs(o) + RAD_ATOL
    viol = (err > tol) & ok[..., None]
    rel = err / np.maximum(np.abs(o), 1e-12)
    info = dict(max_rel=float(rel[ok].max()) if ok.any() else 0.0,
                p999_rel=float(np.quantile(rel[ok], 0.999)) if ok.any() else 0.0,
                checked=int(ok.sum()), excluded=int(bad.sum()), excluded_frac=float(bad.mean()))
    assert not viol.any(), f"{int(viol.sum())} channel values off; worst at {np.argwhere(viol)[:5]}; {info}"
    return info


def segments_by_key(si, sf=None):
    """{(sample, node): (tri, flags)}"""
    out = {}
    for r in np.asarray(si):
        out[(int(r[0]), int(r[1]))] = (int(r[2]), int(r[3]))
    return out


def assert_hit_id_parity(seg_gpu_i, orc, spp, view_offset=0):
    """Every (sample, heap node) of a non-degenerate pixel: same set of
    segments and the same hit triangle, bit for bit."""
    bad = degenerate_pixels(orc).reshape(-1)
    o = segments_by_key(orc["seg_i"])
    g = {}
    for r in np.asarray(seg_gpu_i):
        g[(int(r[0]) - view_offset, int(r[1]))] = (int(r[2]), int(r[3]))
    ok_keys_o = {k for k in o if not bad[k[0] // spp]}
    ok_keys_g = {k for k in g if 0 <= k[0] // spp < bad.size and not bad[k[0] // spp]}
    assert ok_keys_o == ok_keys_g, (f"segment sets differ: only oracle {sorted(ok_keys_o - ok_keys_g)[:5]}, "
                                    f"only gpu {sorted(ok_keys_g - ok_keys_o)[:5]}")
    mism = [(k, o[k], g[k]) for k in ok_keys_o if o[k][0] != g[k][0]]
    assert not mism, f"{len(mism)} hit ids differ, e.g. {mism[:5]}"
    # flags that define the tree (inside, TIR, backfacing, discarded, miss) agree too
    mask = O.SEG_INSIDE | O.SEG_TIR | O.SEG_BACKFACING | O.SEG_DISCARDED | O.SEG_MISS
    fm = [(k, o[k][1] & mask, g[k][1] & mask) for k in ok_keys_o if (o[k][1] & mask) != (g[k][1] & mask)]
    assert not fm, f"{len(fm)} event flags differ, e.g. {fm[:5]}"
    return len(ok_keys_o)
