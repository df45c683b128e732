"""Traversal order (tuning trace_order = b key bits): every level after the
camera rays is traced bucket by bucket, the bucket being the top b bits of a
per-segment key (direction octant, then the Morton code of the origin; the
scene index first in a batch), counted while the level is shaded into
existence and turned into an order by one scan in the level's own
not-yet-written hit and flag words.  The order changes nothing that is
traced: the same segments, hits, flags and node visits as in append order,
and the same images and gradients, for one scene at several key widths, a
batch (scene index in the bucket), a checkpointed tape, and levels of a few
segments."""
import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GpuScene, assert_radiance_parity

pytestmark = pytest.mark.gpu
ORDER = 20  # key bits of the traversal-order buckets (the default)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()
    old = dt.get_tuning()
    dt.set_tuning(order_min_rays=0)  # these small renders are ordered too
    yield
    dt.set_tuning(**old)


def _genus2(w=64, h=64, views=2, depth=8, checkpoint=False):
    V, F = S.two_tori_mesh(48)
    gs = GpuScene(V, F, 1.5, np.array([0.3, 0.1, 0.05], np.float32), S.sh_env_map(64, 32, 1),
                  S.fibonacci_views(views, 3.0, w, h), w, h, depth, spp=2, jitter=1, seed=9)
    if checkpoint:
        p = gs.params
        gs.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, checkpoint=True)
    return gs


def _run(gs, order, g=None):
    dt.set_tuning(trace_order=order)
    dt.profile_read()
    dt.profile_enable(True)
    try:
        img, tape = gs.render()
        grads = dt.render_backward(tape, g) if g is not None else None
        torch.cuda.synchronize()
    finally:
        dt.profile_enable(False)
    prof = dt.profile_read()
    return img, tape, grads, prof


def _sorts(prof, depth):
    """one sort per level after the camera rays, per forward (a render that
    outgrew its workspace runs again)"""
    n = prof.get("k_order", (0, 0.0))[0]
    return n > 0 and n % depth == 0


def _sorted_dump(tape):
    si, sf = dt.dump_segments(tape)
    si, sf = si.cpu().numpy(), sf.cpu().numpy()
    key = np.lexsort((si[:, 1], si[:, 0]))  # arena order depends on CTA scheduling: sort by (sample, node)
    return si[key], sf[key]


@pytest.mark.parametrize("bits", [12, ORDER, 22])
def test_order_finds_the_same_hits(bits):
    gs = _genus2()
    img0, tape0, _, prof0 = _run(gs, 0)
    img1, tape1, _, prof1 = _run(gs, bits)
    s0, s1 = tape0.stats, tape1.stats
    assert s0["status"] == s1["status"] == dt.DT_OK
    for key in ("segments", "level_count", "hits", "misses", "tir", "nodes_visited", "tris_tested"):
        assert s0[key] == s1[key], key
    si0, sf0 = _sorted_dump(tape0)
    si1, sf1 = _sorted_dump(tape1)
    np.testing.assert_array_equal(si0, si1)
    np.testing.assert_array_equal(sf0, sf1)
    np.testing.assert_allclose(img1.cpu().numpy(), img0.cpu().numpy(), rtol=1e-6, atol=1e-7)
    # the sorted path ran: one sort per level after the camera rays
    assert "k_order" not in prof0
    assert _sorts(prof1, gs.params.max_depth)
    assert_radiance_parity(img1[0], gs.oracle(0), 0.103)


def test_order_gives_the_same_gradients():
    gs = _genus2(48, 40)
    rng = np.random.default_rng(3)
    g = torch.from_numpy(rng.normal(size=(2, 40, 48, 3)).astype(np.float32)).cuda()
    _, _, (dV0, di0, ds0), _ = _run(gs, 0, g)
    _, _, (dV1, di1, ds1), _ = _run(gs, ORDER, g)
    a, b = dV0.cpu().numpy().astype(np.float64), dV1.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    assert float(di1) == pytest.approx(float(di0), rel=1e-5, abs=1e-8)
    np.testing.assert_allclose(ds1.cpu().numpy(), ds0.cpu().numpy(), rtol=1e-5, atol=1e-8)


def test_order_in_a_checkpointed_tape():
    gs = _genus2(48, 40, checkpoint=True)
    rng = np.random.default_rng(4)
    g = torch.from_numpy(rng.normal(size=(2, 40, 48, 3)).astype(np.float32)).cuda()
    img0, tape0, (dV0, di0, _), _ = _run(gs, 0, g)
    img1, tape1, (dV1, di1, _), prof = _run(gs, ORDER, g)
    assert tape1.ws.level_capacity > 0 and _sorts(prof, gs.params.max_depth)
    assert tape0.stats["nodes_visited"] == tape1.stats["nodes_visited"]
    np.testing.assert_allclose(img1.cpu().numpy(), img0.cpu().numpy(), rtol=1e-6, atol=1e-7)
    a, b = dV0.cpu().numpy().astype(np.float64), dV1.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    assert float(di1) == pytest.approx(float(di0), rel=1e-5, abs=1e-8)


def test_order_in_a_batch():
    """Two scenes in one table: the keys carry the scene index (four passes)."""
    sc = S.glass_icosphere_scene(width=24, height=24)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 24, 24, 5)
    scenes = [_genus2(32, 32, depth=6), ico]
    items = [dt.BatchItem(g.V, g.F, g.bvh, g.N, g.ior, g.sigma, g.env, g.cams, g.width, g.height, g.params)
             for g in scenes]
    rng = np.random.default_rng(5)
    grads = [torch.from_numpy(rng.normal(size=(g.cams.shape[0], g.height, g.width, 3)).astype(np.float32)).cuda()
             for g in scenes]
    out = {}
    for order in (0, ORDER):
        dt.set_tuning(trace_order=order)
        imgs, tape = dt.render_batch(items)
        out[order] = ([i.cpu().numpy() for i in imgs], tape.stats, dt.render_batch_backward(tape, grads))
    (i0, s0, g0), (i1, s1, g1) = out[0], out[ORDER]
    assert s0["segments"] == s1["segments"] and s0["nodes_visited"] == s1["nodes_visited"]
    for a, b in zip(i0, i1):
        np.testing.assert_allclose(b, a, rtol=1e-6, atol=1e-7)
    for (dVa, dia, _), (dVb, dib, _) in zip(g0, g1):
        a, b = dVa.cpu().numpy().astype(np.float64), dVb.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(a), 1e-12)
        assert float(dib) == pytest.approx(float(dia), rel=1e-5, abs=1e-8)


def test_order_with_tiny_levels():
    """Levels of a few segments: most CTAs of the sort get empty chunks."""
    sc = S.glass_icosphere_scene(width=3, height=2)
    gs = GpuScene.from_scene(sc, max_depth=6)
    img0, tape0, _, _ = _run(gs, 0)
    img1, tape1, _, prof = _run(gs, ORDER)
    assert _sorts(prof, 6) and tape1.stats["status"] == dt.DT_OK
    np.testing.assert_array_equal(_sorted_dump(tape0)[0], _sorted_dump(tape1)[0])
    assert_radiance_parity(img1[0], gs.oracle(0), 0.3333)  # 2 of its 6 pixels


def test_small_renders_keep_append_order():
    """Below order_min_rays camera rays a render traces in append order (no
    order launches) and finds the same hits as with the order."""
    old = dt.get_tuning()
    try:
        gs = GpuScene.from_scene(S.glass_icosphere_scene(width=32, height=32))
        dt.set_tuning(order_min_rays=32 * 32 + 1)
        img0, tape0, _, prof0 = _run(gs, ORDER)
        dt.set_tuning(order_min_rays=0)
        img1, tape1, _, prof1 = _run(gs, ORDER)
        assert "k_order" not in prof0 and _sorts(prof1, gs.params.max_depth)
        np.testing.assert_array_equal(_sorted_dump(tape0)[0], _sorted_dump(tape1)[0])
        np.testing.assert_allclose(img1.cpu().numpy(), img0.cpu().numpy(), rtol=1e-6, atol=1e-7)
    finally:
        dt.set_tuning(**old)
