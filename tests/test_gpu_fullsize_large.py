"""The large optimisation step at full size, in the launch configuration of
bench.py's large leg: a noisy sphere of about 1.06M triangles (marching
tetrahedra on 240^3), one 800x800 view with 8 jittered samples per pixel,
depth 16, IoR 1.52, sigma (0.3, 0.1, 0.05), a 2048x1024 environment,
binned-SAH BVH.

On this noisy surface a path is chaotic after a few bounces: tilting its
camera ray by 1e-6 rad changes a later event or moves a later throughput by
more than 1e-4, so FP32 and FP64 trees part there (measured with the oracle
on 400 seeded pixels: 99 of 273 depth-3 segments keep their events under
the tilt and 34 their throughput and contribution, 4 of 274 at depth 5 their
events, none deeper).  The checks are
therefore: (1) the checkpointed 8-sample render's statistics, and its image
mean against a 1-sample render of the same configuration; (2) on the
1-sample, depth-16 render, every segment at every depth whose path up to it
is stable -- no degenerate event, the same events (and, for the weights,
throughputs and contributions within 1e-4) when the camera ray is tilted
by 1e-6 rad four ways -- against the
oracle's tree: the same segments, hit triangles, events, throughput W and
escaped contribution W * E(d); (3) one-step parity at every depth 0..16:
for seeded segments of each depth the oracle traces one step from the GPU's
own FP32 segment, which the GPU's hit, events and children must match (the
FP32 error does not compound along the path there); (4) at depth 3 (same
mesh, environment, camera, samples), the radiance of sampled stable pixels
and the gradient of a loss seeded on a few of them (exact IoR and sigma
derivatives, two random directional derivatives in the vertices)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import (GRAD_RTOL, PROBE, RAD_ATOL, RAD_RTOL, assert_segment_weights, sample_segments_by_depth,
                            step_parity)

pytestmark = pytest.mark.gpu

RES, SPP, DEPTH, SEED = 800, 8, 16, 11
IOR, SIGMA = 1.52, np.array([0.3, 0.1, 0.05], np.float32)
SHALLOW = 3
DEGEN = O.SEG_NEAR_EDGE | O.SEG_NEAR_TIE | O.SEG_NEAR_CRITICAL | O.SEG_GRAZING | O.SEG_NEAR_POLE
EVENTS = O.SEG_INSIDE | O.SEG_TIR | O.SEG_BACKFACING | O.SEG_DISCARDED | O.SEG_MISS


@pytest.fixture(scope="module")
def large():
    from paper_2603_00413_gb300 import build
    build.build()
    V, F = S.noisy_sphere_mesh(240, seed=3, amplitude=0.1, octaves=3)
    env = S.sh_env_map(2048, 1024, 3)
    cam = S.camera((0.45, 0.35, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, RES, RES)
    dev = torch.device("cuda:0")
    Vt, Ft = torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev)
    scene = (Vt, Ft, dt.build_bvh(Vt, Ft), dt.vertex_normals(Vt, Ft), torch.tensor([IOR], device=dev),
             torch.from_numpy(SIGMA).to(dev), torch.from_numpy(env).to(dev),
             torch.from_numpy(cam.as_array()[None]).to(dev))
    o, d = O.camera_rays(cam, 1, 1, SEED, 0)
    return dict(V=V, F=F, env=env, scene=scene, o=o, d=d)


def _render(L, depth, spp, checkpoint):
    p = dt.Params(depth, spp=spp, jitter=1, seed=SEED, checkpoint=checkpoint)
    return dt.render(*L["scene"], RES, RES, p)


def test_large_eight_sample_checkpointed_render(large):
    img8, tape8 = _render(large, DEPTH, SPP, True)
    st = tape8.stats
    assert st["status"] == dt.DT_OK and st["n_levels"] == DEPTH + 1
    assert st["level_count"][0] == RES * RES * SPP
    assert tape8.ws.level_capacity >= st["level_needed"]
    m8 = img8.double().mean(dim=(0, 1, 2)).cpu().numpy()
    del tape8, img8
    img1, _ = _render(large, DEPTH, 1, True)
    m1 = img1.double().mean(dim=(0, 1, 2)).cpu().numpy()
    # two estimates of the same pixel integrals (jittered sub-pixel positions)
    np.testing.assert_allclose(m8, m1, rtol=2e-2)


def _tilted(d, eps):
    """d turned by eps radians four ways (two orthogonal planes, both signs)"""
    a = np.where(np.abs(d[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    u = np.cross(d, a)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(d, u)
    out = []
    for w in (u, -u, v, -v):
        t = d + eps * w
        out.append(t / np.linalg.norm(t, axis=1, keepdims=True))
    return out


def _segments(L, o, d, pix):
    r = O.render_rays(L["V"], L["F"], IOR, SIGMA, L["env"], o, d, DEPTH, segments=True)
    si = r["seg_i"].copy()
    si[:, 0] = pix[si[:, 0]]  # oracle ray index -> sample index
    return si, r["seg_f"]


@pytest.fixture(scope="module")
def deep(large):
    img, tape = _render(large, DEPTH, 1, False)
    assert tape.stats["status"] == dt.DT_OK and tape.stats["n_levels"] == DEPTH + 1
    si, sf = dt.dump_segments(tape)
    return si, sf


def test_large_stable_prefix_segments_every_depth(large, deep):
    si, sf = deep
    rng = np.random.default_rng(21)
    pix = np.unique(rng.integers(0, RES * RES, size=400))
    sel = torch.isin(si[:, 0], torch.from_numpy(pix.astype(np.int32)).cuda())
    g_i, g_f = si[sel].cpu().numpy(), sf[sel].cpu().numpy()
    o, d = large["o"][pix], large["d"][pix]
    osi, osf = _segments(large, o, d, pix)
    base = {(int(a), int(n)): (int(t), int(f) & EVENTS, osf[j, 9:15]) for j, (a, n, t, f) in enumerate(osi)}
    flags = {(int(a), int(n)): int(f) for a, n, _, f in osi}
    tilts = []
    for dt_ in _tilted(d, PROBE):
        ti, tf = _segments(large, o, dt_, pix)
        tilts.append({(int(a), int(n)): (int(t), int(f) & EVENTS, tf[j, 9:15]) for j, (a, n, t, f) in enumerate(ti)})

    def step_stable(k, weights):
        if flags[k] & DEGEN:
            return False
        b = base[k]
        for tv in tilts:
            x = tv.get(k)
            if x is None or x[:2] != b[:2]:
                return False
            if weights and np.any(np.abs(x[2] - b[2]) > RAD_RTOL * np.abs(b[2]) + RAD_ATOL):
                return False
        return True

    memo = {}

    def stable(k, weights):
        m = k[1]
        while m >= 1:
            km = (k[0], m, weights)
            if km not in memo:
                memo[km] = step_stable((k[0], m), weights)
            if not memo[km]:
                return False
            m //= 2
        return True

    ev_keys = [k for k in base if stable(k, False)]
    w_keys = [k for k in base if stable(k, True)]
    g_all = {(int(a), int(n)): (int(t), int(f) & EVENTS) for a, n, t, f in g_i}
    # every event-stable oracle segment exists on the GPU with the same hit and events
    missing = [k for k in ev_keys if k not in g_all]
    assert not missing, missing[:5]
    diff = [(k, base[k][:2], g_all[k]) for k in ev_keys if g_all[k] != base[k][:2]]
    assert not diff, diff[:5]
    # and below an event-stable parent the GPU has no segment the oracle lacks
    ev_set = set(ev_keys)
    extra = [k for k in g_all if k not in base and k[1] > 1 and (k[0], k[1] // 2) in ev_set]
    assert not extra, extra[:5]
    # throughput and escaped contribution of the weight-stable ones
    assert_segment_weights(g_i, g_f, osi, osf, w_keys)

    def per_depth(keys):
        return np.bincount([int(np.floor(np.log2(k[1]))) for k in keys], minlength=DEPTH + 1)

    ev_n, w_n, all_n = per_depth(ev_keys), per_depth(w_keys), per_depth(list(base))
    print("segments checked per depth (events / throughput / all):",
          [f"{a}/{b}/{c}" for a, b, c in zip(ev_n, w_n, all_n)])
    # measured with the oracle alone: events 399/342/226/99/31/4 at depths
    # 0-5, throughputs and contributions 399/250/128/34/7, none deeper
    assert ev_n[0] >= 390 and ev_n[3] >= 80 and w_n[2] >= 100 and w_n[3] >= 25, (ev_n.tolist(), w_n.tolist())


def test_large_step_parity_every_depth(large, deep):
    si, sf = deep
    rows = sample_segments_by_depth(si, 300, DEPTH, seed=24)
    # the noisy surface's sharp folds make more steps ill-conditioned (7.2 %
    # measured) than the smooth meshes' 1-3 %
    info = step_parity(si, sf, rows, large["V"], large["F"], IOR, SIGMA, large["env"], DEPTH, max_unconditioned=0.092)
    print("one-step parity:", info)
    per = info["checked_per_depth"]
    # every level of the depth-16 tree holds far more than 300 segments; at
    # most a quarter of a level's are ill-conditioned (measured: 227 of the
    # 300 camera rays checked, 274-300 at the later depths)
    assert min(per) >= 200, per


def _stable_pixels(L, n, seed, depth):
    """n seeded pixels whose path hits the object and is not edge-degenerate
    at the given depth (drawn in rounds of candidates)."""
    rng = np.random.default_rng(seed)
    got = []
    for _ in range(8):
        cand = rng.integers(0, RES * RES, size=3 * n)
        r = O.render_rays(L["V"], L["F"], IOR, SIGMA, L["env"], L["o"][cand], L["d"][cand], depth, probe=PROBE,
                          segments=True)
        hit = np.zeros(len(cand), bool)
        hit[np.unique(r["seg_i"][r["seg_i"][:, 2] >= 0, 0])] = True
        ok = hit & ((r["pix_flags"] & O.SEG_DEGENERATE) == 0)
        got += [(int(p), r["img"][i]) for i, p in enumerate(cand) if ok[i]]
        if len(got) >= n:
            break
    assert len(got) >= n, len(got)
    return got[:n]


def test_large_shallow_radiance_and_gradient(large):
    img, tape = _render(large, SHALLOW, 1, True)
    got = _stable_pixels(large, 12, 22, SHALLOW)
    pix = np.array([p for p, _ in got])
    g = img.view(-1, 3)[torch.from_numpy(pix).cuda()].cpu().numpy().astype(np.float64)
    ref = np.stack([v for _, v in got])
    err = np.abs(g - ref)
    assert (err <= RAD_RTOL * np.abs(ref) + RAD_ATOL).all(), (err / np.maximum(np.abs(ref), 1e-12)).max()
    # gradient of a loss seeded on four of them
    pix = pix[:4]
    rng = np.random.default_rng(23)
    gp = rng.normal(size=(len(pix), 3))
    grad = torch.zeros(RES * RES, 3, device="cuda")
    grad[torch.from_numpy(pix).cuda()] = torch.from_numpy(gp.astype(np.float32)).cuda()
    dV, dior, dsig = dt.render_backward(tape, grad.view(1, RES, RES, 3))
    nv = large["V"].shape[0]
    U = rng.normal(size=(2, nv, 3))
    tV = np.concatenate([np.zeros((4, nv, 3)), U])
    tior = np.array([1.0, 0, 0, 0, 0, 0])
    tsig = np.zeros((6, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    _, dimg = O.render_rays_jvp(large["V"], large["F"], IOR, SIGMA, large["env"], large["o"][pix], large["d"][pix],
                                SHALLOW, tV, tior, tsig)
    J = np.einsum("knc,nc->k", dimg, gp)
    assert float(dior) == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1.0, abs(J[0])))
    np.testing.assert_allclose(dsig.cpu().numpy(), J[1:4], rtol=GRAD_RTOL, atol=1e-6 * max(1.0, np.abs(J[1:4]).max()))
    dVg = dV.cpu().numpy().astype(np.float64)
    for j in range(2):
        proj = float((dVg * U[j]).sum())
        # |<e, u>| ~ |e| for u ~ N(0, I): bounded against the gradient's norm
        assert abs(proj - J[4 + j]) <= GRAD_RTOL * abs(J[4 + j]) + 3 * GRAD_RTOL * np.linalg.norm(dVg), (proj, J[4 + j])
