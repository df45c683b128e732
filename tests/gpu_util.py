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


# Each parity test states the fraction of its pixels that the oracle's
# criterion excludes (measured with the oracle alone on the test's scene),
# and fails when the fraction grows past it by more than this margin: the
# excluded set may move by a few pixels between hosts (their libm), but a
# change that widens the exclusion cannot hide behind a loose bound.
EXCLUDED_MARGIN = 0.02


def degenerate_pixels(orc):
    return (orc["pix_flags"] & O.SEG_DEGENERATE) != 0


def excluded_pixels(orc, expected, what="view"):
    """The pixels excluded from parity (degenerate_pixels), after checking
    that their fraction is at most the measured `expected` + EXCLUDED_MARGIN."""
    bad = degenerate_pixels(orc)
    frac = float(bad.mean())
    assert frac <= expected + EXCLUDED_MARGIN, (
        f"{what}: {frac:.4f} of the pixels excluded from parity; measured {expected:.4f} "
        f"(+ {EXCLUDED_MARGIN} allowed)")
    return bad


def assert_radiance_parity(img_gpu, orc, expected_excluded, exclude=None):
    """Per pixel and channel |gpu - oracle| <= RAD_RTOL |oracle| + RAD_ATOL on
    pixels whose oracle path has no degenerate event; the fraction of
    excluded pixels must stay within EXCLUDED_MARGIN of expected_excluded."""
    g = img_gpu.detach().cpu().numpy().astype(np.float64)
    o = orc["img"]
    bad = excluded_pixels(orc, expected_excluded)
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
    segments and the same hit triangle, bit for bit, and the same events."""
    bad = degenerate_pixels(orc).reshape(-1)
    o = segments_by_key(orc["seg_i"])
    g = {}
    gi = np.asarray(seg_gpu_i)
    for r in gi:
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


def weight_stable_tree(V, F, ior, sigma, env, o, d, max_depth, t_min=1e-5, medium=None):
    """The oracle's tree of the primary rays (o, d) and the keys (ray, heap
    node) of its segments whose path up to and including them is stable:
    no degenerate event, and with the primary ray tilted by PROBE four ways
    the same segment, hit and events, and a throughput and escaped
    contribution within the radiance tolerance.  A pixel's radiance sums many segments, so one segment's
    throughput can move more under the tilt than the pixel does: the
    per-segment comparison needs the per-segment criterion."""
    def tree(dd):
        r = O.render_rays(V, F, ior, sigma, env, o, dd, max_depth, t_min, segments=True, medium=medium)
        return r["seg_i"], r["seg_f"]

    bi, bf = tree(d)
    base = {(int(a), int(n)): (int(t), int(f) & EVENTS, bf[j, 9:15]) for j, (a, n, t, f) in enumerate(bi)}
    flags = {(int(a), int(n)): int(f) for a, n, _, f in bi}
    tilts = []
    for dq in tilted_directions(np.asarray(d, np.float64), PROBE):
        ti, tf = tree(dq)
        tilts.append({(int(a), int(n)): (int(t), int(f) & EVENTS, tf[j, 9:15]) for j, (a, n, t, f) in enumerate(ti)})
    degen = O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE | O.SEG_NEAR_CRITICAL | O.SEG_GRAZING | O.SEG_NEAR_POLE
    memo = {}

    def ok(k):
        if k not in memo:
            b = base[k]
            good = not flags[k] & degen
            for tv in tilts:
                x = tv.get(k)
                good = good and x is not None and x[:2] == b[:2] and bool(
                    np.all(np.abs(x[2] - b[2]) <= RAD_RTOL * np.abs(b[2]) + RAD_ATOL))
            memo[k] = good
        return memo[k]

    def stable(k):
        m = k[1]
        while m >= 1:
            if not ok((k[0], m)):
                return False
            m //= 2
        return True

    return bi, bf, [k for k in base if stable(k)]


def assert_tree_weights(gs, view, seg_gpu_i, seg_gpu_f, expected_unstable, medium=None):
    """Throughput and escaped contribution of every weight-stable segment of
    one view of a GpuScene against the oracle's tree (weight_stable_tree);
    the fraction of segments left out is bounded by its measured value."""
    p = gs.params
    o, d = O.camera_rays(gs.cam_list[view], p.spp, p.jitter, p.seed, view)
    bi, bf, keys = weight_stable_tree(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, o, d, p.max_depth, p.t_min,
                                      medium=medium)
    frac = 1.0 - len(keys) / max(len(bi), 1)
    assert frac <= expected_unstable + EXCLUDED_MARGIN, (frac, expected_unstable)
    npix_spp = gs.width * gs.height * p.spp
    n = assert_segment_weights(np.asarray(seg_gpu_i), np.asarray(seg_gpu_f), bi, bf, keys, view * npix_spp)
    return n, frac


def assert_segment_weights(gi, gf, oi, of, keys, view_offset=0):
    """Throughput W (columns 9-11) and escaped contribution W * E(d)
    (columns 12-14) of the segments `keys` ((sample, node) pairs, the
    sample in the oracle's numbering): GPU (FP32) within RAD_RTOL relative
    + RAD_ATOL of the oracle (FP64).  Returns the number compared."""
    gpos = {(int(r[0]) - view_offset, int(r[1])): j for j, r in enumerate(gi)}
    opos = {(int(r[0]), int(r[1])): j for j, r in enumerate(oi)}
    ks = sorted(keys)
    if not ks:
        return 0
    a = gf[[gpos[k] for k in ks]][:, 9:15].astype(np.float64)
    b = of[[opos[k] for k in ks]][:, 9:15]
    err = np.abs(a - b)
    viol = err > RAD_RTOL * np.abs(b) + RAD_ATOL
    if viol.any():
        rows = np.nonzero(viol.any(axis=1))[0]
        ex = [(ks[r], a[r].tolist(), b[r].tolist()) for r in rows[:3]]
        raise AssertionError(f"{len(rows)} of {len(ks)} segments' throughput or contribution off, e.g. {ex}")
    return len(ks)


# ---------------------------------------------------------------------------
# one-step parity at every depth
# ---------------------------------------------------------------------------
EVENTS = O.SEG_INSIDE | O.SEG_TIR | O.SEG_BACKFACING | O.SEG_DISCARDED | O.SEG_MISS
# a step whose hit lies within 1e-6 of an edge or near-ties another: its hit
# id is not defined to FP32 (hit ids are compared bit for bit only away from
# edges)
STEP_EDGE = O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE
# a step whose inside/outside, TIR or backfacing decision, or whose
# environment lookup, sits within 1e-6 of its threshold
STEP_DEGEN = STEP_EDGE | O.SEG_NEAR_CRITICAL | O.SEG_GRAZING | O.SEG_NEAR_POLE


class SegmentIndex:
    """Rows of a GPU segment dump by (sample, heap node), on the device."""

    def __init__(self, si):
        self.si = si
        self.key = (si[:, 0].long() << 32) | si[:, 1].long()
        self.order = torch.argsort(self.key)
        self.skey = self.key[self.order]

    def rows(self, sample, node):
        q = (sample.long() << 32) | node.long()
        pos = torch.searchsorted(self.skey, q).clamp_(max=max(self.skey.numel() - 1, 0))
        return torch.where(self.skey[pos] == q, self.order[pos], torch.full_like(pos, -1))


def sample_segments_by_depth(si, per_depth, max_depth, seed):
    """Up to per_depth rows of each depth 0..max_depth (depth = floor(log2
    node)), drawn with a seeded generator from the rows in (sample, node)
    order, so that the same segments are drawn whatever order the device
    appended them in; returns a device index tensor."""
    key = (si[:, 0].long() << 32) | si[:, 1].long()
    by_key = torch.argsort(key)
    node = si[by_key, 1].long()
    depth = torch.floor(torch.log2(node.double())).long()
    gen = torch.Generator(device=si.device)
    gen.manual_seed(seed)
    out = []
    for k in range(max_depth + 1):
        rows = by_key[torch.nonzero(depth == k).flatten()]
        if rows.numel() > per_depth:
            rows = rows[torch.randperm(rows.numel(), generator=gen, device=si.device)[:per_depth]]
        out.append(rows)
    return torch.cat(out)


def tilted_directions(d, eps):
    """d turned by eps radians four ways (two orthogonal planes, both signs),
    as the oracle's stability probe turns a camera ray."""
    a = np.where(np.abs(d[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    u = np.cross(d, a)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(d, u)
    out = []
    for w in (u, -u, v, -v):
        t = d + eps * w
        out.append(t / np.linalg.norm(t, axis=1, keepdims=True))
    return out


def _step_conditioned(ti, tf, tilts):
    """Steps whose outcome is stable under the probe: for every tilted copy
    of the segment's direction, the same hit, events and children, and the
    children's throughputs, an escape's contribution (both within the
    radiance tolerance) and the children's directions (within 1e-4) barely
    move.  A FP32 direction carries ~1e-7 of error, a tenth of the tilt, so
    on these steps the FP32 result stays within the tolerances; the others
    (chiefly refraction close to the critical angle, where T = 1 - R and
    the refracted direction change fast) are excluded like an edge."""
    ok = np.ones(ti.shape[0], bool)
    for qi, qf in tilts:
        ok &= (qi[:, 0, 2] == ti[:, 0, 2]) & ((qi[:, 0, 3] & EVENTS) == (ti[:, 0, 3] & EVENTS))
        ok &= (qi[:, 1:, 1] == ti[:, 1:, 1]).all(axis=1)
        w, wq = tf[:, :, 9:15], qf[:, :, 9:15]
        ok &= (np.abs(wq - w) <= RAD_RTOL * np.abs(w) + RAD_ATOL).all(axis=(1, 2))
        ok &= (np.abs(qf[:, 1:, 6:9] - tf[:, 1:, 6:9]) <= 1e-4).all(axis=(1, 2))
    return ok


def step_parity(si, sf, rows, V, F, ior, sigma, env, max_depth, t_min=1e-5, medium=None, dir_tol=5e-5,
                pos_tol=2e-5, max_unconditioned=0.05):
    """One-step parity of GPU segments at any depth.  For each dump row in
    `rows` the oracle traces one step in FP64 from the GPU's own segment (its
    FP32 origin and direction, the triangle it leaves -- its parent's hit --
    and its depth) and the GPU's record must agree: the hit triangle bit for
    bit (except within 1e-6 of an edge), the events (except near a decision
    threshold), which children exist, each child's origin and direction
    within pos_tol and dir_tol (a well-conditioned step moves a child's
    direction by at most 1e-4 under a 1e-6 rad tilt, 100 times its input;
    the GPU's FP32 origin and direction carry ~1e-7 to ~2e-7 of error, which
    also shifts the interpolated normal on a small triangle, so the children's
    directions may differ by a few 1e-5: measured up to 2.2e-5 on the noisy
    sphere), each child's throughput relative to its
    parent's within the radiance tolerance, and an escaped segment's
    contribution relative to its throughput the same -- on the steps that
    are well conditioned (_step_conditioned; at most max_unconditioned of
    them are not).  A step starts from the same inputs on both sides, so
    the FP32 error does not grow with the depth and every level of the tree
    is checked.  si, sf: the dump (device tensors); returns dict of
    per-depth counts and the largest errors."""
    idx = SegmentIndex(si)
    rows = rows.to(si.device)
    s, m = si[rows, 0], si[rows, 1]
    parent = idx.rows(s, torch.div(m, 2, rounding_mode="floor"))
    kid_r, kid_t = idx.rows(s, 2 * m), idx.rows(s, 2 * m + 1)
    src = torch.where((m > 1) & (parent >= 0), si[parent.clamp(min=0), 2], torch.full_like(m, -1))
    assert bool(((m == 1) | (parent >= 0)).all()), "a sampled segment's parent is missing from the dump"
    g_i = si[rows].cpu().numpy()
    g_f = sf[rows].cpu().numpy().astype(np.float64)
    kids = [k.cpu().numpy() for k in (kid_r, kid_t)]
    kid_f = [sf[k.clamp(min=0)].cpu().numpy().astype(np.float64) for k in (kid_r, kid_t)]
    depth = np.floor(np.log2(g_i[:, 1].astype(np.float64))).astype(int)
    src_np = src.cpu().numpy()
    ti, tf = O.trace_steps(V, F, ior, sigma, env, g_f[:, 3:6], g_f[:, 6:9], src_np, depth, max_depth, t_min,
                           medium=medium)
    tilts = [O.trace_steps(V, F, ior, sigma, env, g_f[:, 3:6], dq, src_np, depth, max_depth, t_min, medium=medium)
             for dq in tilted_directions(g_f[:, 6:9], PROBE)]
    of = ti[:, 0, 3]
    edge = (of & STEP_EDGE) != 0
    unc = ~_step_conditioned(ti, tf, tilts)
    degen = ((of & STEP_DEGEN) != 0) | unc
    assert unc.mean() <= max_unconditioned, f"{unc.mean():.4f} of the steps are ill-conditioned"
    # a step whose hit changes when its direction is tilted by the probe
    # (within FP32 resolution of an edge: a far ray's FP32 barycentrics carry
    # ~1e-5 of error on a small triangle) is edge-degenerate for its hit id
    # too, as the pixel probe of c21 makes it for a path
    bad_tri = ~edge & ~unc & (ti[:, 0, 2] != g_i[:, 2])
    if bad_tri.any():
        ex = []
        for j in np.nonzero(bad_tri)[0][:3]:
            # the oracle's distance to each of the two triangles from the GPU's own segment
            tt = []
            for f in (int(ti[j, 0, 2]), int(g_i[j, 2])):
                if f < 0:
                    tt.append(None)
                    continue
                r = O.closest_hit(V, np.asarray(F)[[f]], g_f[j:j + 1, 3:6], g_f[j:j + 1, 6:9], None, t_min)
                tt.append((float(r[1][0]), float(r[2][0]), float(r[3][0]), int(r[4][0])))
            ex.append(dict(gpu=g_i[j].tolist(), gpu_t=float(g_f[j, 0]), src=int(src_np[j]), oracle_tri=int(ti[j, 0, 2]),
                           oracle_flags=int(of[j]), t_b1_b2_flags=tt, o=g_f[j, 3:6].tolist(), d=g_f[j, 6:9].tolist()))
        raise AssertionError(f"{int(bad_tri.sum())} of {len(rows)} steps hit another triangle: {ex}")
    ok = ~degen
    bad_ev = ok & ((of & EVENTS) != (g_i[:, 3] & EVENTS))
    assert not bad_ev.any(), (f"{int(bad_ev.sum())} steps differ in events, e.g. "
                              f"{[(g_i[j].tolist(), int(of[j])) for j in np.nonzero(bad_ev)[0][:3]]}")
    worst = dict(dir=0.0, pos=0.0, w=0.0, c=0.0)
    # ratios need a normal FP32 throughput (deep paths of strongly absorbing
    # glass fall into the subnormal range, where FP32 keeps few bits)
    wok = g_f[:, 9:12].min(axis=1) > 1e-30
    for c in (1, 2):
        g_has = kids[c - 1] >= 0
        o_has = ti[:, c, 1] != 0
        diff = ok & (g_has != o_has)
        assert not diff.any(), f"{int(diff.sum())} steps differ in whether child {c} exists"
        both = ok & g_has & o_has
        kf = kid_f[c - 1][both]
        orc = tf[both, c]
        e_pos = np.abs(kf[:, 3:6] - orc[:, 3:6]).max(axis=1, initial=0.0)
        e_dir = np.abs(kf[:, 6:9] - orc[:, 6:9]).max(axis=1, initial=0.0)
        wb = wok[both]
        w_rel = kf[wb, 9:12] / g_f[both][wb, 9:12]
        e_w = (np.abs(w_rel - orc[wb, 9:12]) / (np.abs(orc[wb, 9:12]) + RAD_ATOL)).max(axis=1, initial=0.0)
        worst["pos"] = max(worst["pos"], float(e_pos.max(initial=0.0)))
        worst["dir"] = max(worst["dir"], float(e_dir.max(initial=0.0)))
        worst["w"] = max(worst["w"], float(e_w.max(initial=0.0)))
        assert (e_pos <= pos_tol).all() and (e_dir <= dir_tol).all(), (c, worst)
        assert (e_w <= RAD_RTOL).all(), (c, worst)
    miss = ok & wok & ((g_i[:, 3] & O.SEG_MISS) != 0)
    c_rel = g_f[miss, 12:15] / g_f[miss, 9:12]
    e_c = (np.abs(c_rel - tf[miss, 0, 12:15]) / (np.abs(tf[miss, 0, 12:15]) + RAD_ATOL)).max(axis=1, initial=0.0)
    worst["c"] = float(e_c.max(initial=0.0))
    assert (e_c <= RAD_RTOL).all(), worst
    per_depth = np.bincount(depth[ok], minlength=max_depth + 1)
    return dict(checked_per_depth=per_depth.tolist(), excluded=int(degen.sum()), ill_conditioned=int(unc.sum()),
                hit_ids=int((~edge).sum()), worst=worst)
