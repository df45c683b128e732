"""Batched rendering: scenes of uneven size, depth, sample count and
material in one render give the same images, segments and gradients as each
scene rendered alone, and a batch captured in a CUDA graph replays to the
same result.  (Float atomics accumulate images and gradients, so results
agree to rounding, not bit for bit; paths and segment counts agree exactly.)"""
import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL
from tests.gpu_util import GpuScene, assert_radiance_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes():
    from paper_2603_00413_gb300 import build
    build.build()
    rng = np.random.default_rng(21)
    out = []
    sc = S.glass_icosphere_scene(width=32, height=32)
    out.append(GpuScene(sc.V, sc.F, 1.5, np.zeros(3, np.float32), sc.env, sc.cams, 32, 32, 4))
    V, F = S.two_tori_mesh(32)
    out.append(GpuScene(V, F, 1.42, np.array([0.9, 0.3, 1.4], np.float32), S.sh_env_map(64, 32, 5),
                        S.fibonacci_views(2, 3.0, 24, 20), 24, 20, 8, spp=2, jitter=1, seed=9))
    V, F = S.mesh_from_field(S.random_blob_field(rng), 3000)
    out.append(GpuScene(V, F, 1.61, np.array([0.2, 1.1, 0.6], np.float32), S.sh_env_map(32, 16, 6),
                        [S.camera((0.5, 2.6, 1.2), width=40, height=28)], 40, 28, 6))
    V = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    out.append(GpuScene(V, F, 1.33, np.zeros(3, np.float32), S.sh_env_map(16, 8, 7),
                        [S.camera((0.1, 0.1, 2.0), (0.1, 0.1, 0), width=8, height=8)], 8, 8, 3))
    return out


def _items(gs_list):
    return [dt.BatchItem(g.V, g.F, g.bvh, g.N, g.ior, g.sigma, g.env, g.cams, g.width, g.height, g.params)
            for g in gs_list]


def test_batch_forward_matches_scenes_alone(scenes):
    alone = [g.render() for g in scenes]
    imgs, tape = dt.render_batch(_items(scenes))
    assert tape.stats["segments"] == sum(t.stats["segments"] for _, t in alone)
    assert tape.stats["hits"] == sum(t.stats["hits"] for _, t in alone)
    for (img_a, _), img_b in zip(alone, imgs):
        np.testing.assert_allclose(img_b.cpu().numpy(), img_a.cpu().numpy(), rtol=1e-5, atol=1e-7)
    assert_radiance_parity(imgs[0][0], scenes[0].oracle(0), 0.0293)


def test_batch_backward_matches_scenes_alone(scenes):
    rng = np.random.default_rng(22)
    grads = [torch.from_numpy(rng.normal(size=(g.cams.shape[0], g.height, g.width, 3)).astype(np.float32)).cuda()
             for g in scenes]
    alone = []
    for g, gr in zip(scenes, grads):
        _, tape = g.render()
        alone.append(dt.render_backward(tape, gr))
    _, btape = dt.render_batch(_items(scenes))
    both = dt.render_batch_backward(btape, grads)
    for (dVa, dia, dsa), (dVb, dib, dsb) in zip(alone, both):
        a, b = dVa.cpu().numpy().astype(np.float64), dVb.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= GRAD_RTOL * max(np.linalg.norm(a), 1e-12)
        assert float(dib) == pytest.approx(float(dia), rel=GRAD_RTOL, abs=1e-7)
        np.testing.assert_allclose(dsb.cpu().numpy(), dsa.cpu().numpy(), rtol=GRAD_RTOL, atol=1e-7)


def test_batch_replays_from_a_cuda_graph(scenes):
    items = _items(scenes)
    imgs, tape = dt.render_batch(items)
    rng = np.random.default_rng(23)
    grads = [torch.from_numpy(rng.normal(size=tuple(i.shape)).astype(np.float32)).cuda() for i in imgs]
    ref = dt.render_batch_backward(tape, grads)
    nbytes = dt.batch_backward_workspace_size(items, tape.stats["max_level"])
    _, bws = dt._aligned_empty(nbytes, imgs[0].device)
    outs = [torch.zeros_like(i) for i in imgs]
    gouts = [(torch.zeros_like(it.V), torch.zeros(1, device="cuda"), torch.zeros(3, device="cuda")) for it in items]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            _, t2 = dt.render_batch(items, ws=tape.ws, outs=outs, check=False)
            t2.stats = tape.stats
            dt.render_batch_backward(t2, grads, bws=bws, outs=gouts)
    for _ in range(2):
        for o in outs:
            o.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        st = dt.read_stats(tape.ws)
        assert st["status"] == dt.DT_OK and st["segments"] == tape.stats["segments"]
        for a, b in zip(imgs, outs):
            np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-5, atol=1e-7)
        for (dVa, dia, dsa), (dVb, dib, dsb) in zip(ref, gouts):
            a, b = dVa.cpu().numpy().astype(np.float64), dVb.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(a - b) <= GRAD_RTOL * max(np.linalg.norm(a), 1e-12)
            assert float(dib) == pytest.approx(float(dia), rel=GRAD_RTOL, abs=1e-7)


def test_batch_rejects_bad_sizes(scenes):
    items = _items(scenes)
    with pytest.raises(dt.DiffTransError):
        dt.render_batch(items * 65)  # 260 entries > 256


def test_autotuner_picks_a_setting_and_results_do_not_change(scenes, tmp_path):
    from paper_2603_00413_gb300 import autotune
    items = _items(scenes)
    ref, tape = dt.render_batch(items)
    outs = [torch.empty_like(r) for r in ref]

    def step():
        dt.render_batch(items, ws=tape.ws, outs=outs, check=False)

    before = dt.get_tuning()
    space = {"bvh_width": (2, 4), "trace_blocks_per_sm": (4, 5), "trace_refill": (4, 16)}
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(step, "test-batch", space=space, reps=1, cache_path=cache, retune=True)
    assert dt.get_tuning() == res["tuning"]
    assert 4 <= len(res["trials"]) <= 1 + 6  # the start, then each knob's other values in turn
    torch.cuda.synchronize()
    for a, b in zip(ref, outs):
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-5, atol=1e-7)
    # cached: a second call sets the same knobs without timing
    dt.set_tuning(**before)
    res2 = autotune.tune(step, "test-batch", space=space, cache_path=cache)
    assert res2["tuning"] == res["tuning"] and dt.get_tuning() == res["tuning"]
    dt.set_tuning(**before)
