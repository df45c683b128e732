"""Per-bounce checkpointing (tape mode 1): the forward keeps every level's ray
queue but only a two-level ring of hit records; the backward recovers each
spawning segment's hit from the source triangle its children carry.
Images, statistics and gradients equal those of the full tape (and the
oracle's), a ring too small for a level is reported and retried, and the
workspace is smaller."""
import copy

import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, GpuScene, assert_radiance_parity, excluded_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def genus2():
    from paper_2603_00413_gb300 import build
    build.build()
    V, F = S.two_tori_mesh(36)
    cams = S.fibonacci_views(2, 3.0, 48, 40)
    return GpuScene(V, F, 1.52, np.array([0.3, 0.1, 0.05], np.float32), S.sh_env_map(64, 32, 1), cams, 48, 40, 8,
                    spp=2, jitter=1, seed=5)


def _checkpointed(gs, level_capacity=0):
    ck = copy.copy(gs)
    p = gs.params
    ck.params = dt.Params(p.max_depth, p.spp, p.jitter, p.seed, p.t_min, checkpoint=True,
                          level_capacity=level_capacity)
    return ck


def _grads(gs, g):
    img, tape = gs.render()
    dV, dior, dsig = dt.render_backward(tape, g)
    return img, tape, dV.cpu().numpy().astype(np.float64), float(dior), dsig.cpu().numpy().astype(np.float64)


def test_checkpointed_forward_equals_full_tape_and_oracle(genus2):
    img_f, tape_f = genus2.render()
    img_c, tape_c = _checkpointed(genus2).render()
    assert tape_c.ws.level_capacity > 0
    assert tape_c.ws.bytes < tape_f.ws.bytes
    for key in ("segments", "hits", "misses", "tir", "backfacing", "level_count", "max_level"):
        assert tape_c.stats[key] == tape_f.stats[key], key
    assert tape_c.stats["level_needed"] == max(tape_f.stats["level_count"])
    np.testing.assert_allclose(img_c.cpu().numpy(), img_f.cpu().numpy(), rtol=1e-6, atol=1e-7)
    assert_radiance_parity(img_c[1], genus2.oracle(1), 0.1656)
    with pytest.raises(ValueError):
        dt.dump_segments(tape_c)


def test_checkpointed_gradients_equal_full_tape(genus2):
    rng = np.random.default_rng(31)
    g = torch.from_numpy(rng.normal(size=(2, genus2.height, genus2.width, 3)).astype(np.float32)).cuda()
    _, _, dVf, diorf, dsigf = _grads(genus2, g)
    dt.profile_read()
    dt.profile_enable(True)
    _, tape_c, dVc, diorc, dsigc = _grads(_checkpointed(genus2), g)
    torch.cuda.synchronize()
    dt.profile_enable(False)
    prof = dt.profile_read()
    # the backward traverses nothing: the hits come from the children's
    # source triangles
    assert "k_trace" not in prof or prof["k_trace"][0] == genus2.params.max_depth + 1
    assert np.linalg.norm(dVc - dVf) <= 1e-4 * np.linalg.norm(dVf)
    assert diorc == pytest.approx(diorf, rel=1e-4, abs=1e-7)
    np.testing.assert_allclose(dsigc, dsigf, rtol=1e-4, atol=1e-7)


def test_checkpointed_gradient_matches_oracle_derivative(genus2):
    """dJ/dIoR and dJ/dsigma of the checkpointed backward against the
    oracle's forward-mode derivative on view 0."""
    import oracle as O
    gs = _checkpointed(genus2)
    rng = np.random.default_rng(32)
    gnp = rng.normal(size=(2, gs.height, gs.width, 3))
    gnp[1] = 0.0
    gnp[0][excluded_pixels(gs.oracle(0), 0.0833)] = 0.0
    _, _, _, dior, dsig = _grads(gs, torch.from_numpy(gnp.astype(np.float32)).cuda())
    p = gs.params
    tior = np.array([1.0, 0, 0, 0])
    tsig = np.zeros((4, 3))
    tsig[1, 0] = tsig[2, 1] = tsig[3, 2] = 1.0
    d = O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, None, tior, tsig, p.spp,
                     p.jitter, p.seed, 0, p.t_min)[1]
    J = np.einsum("khwc,hwc->k", d, gnp[0])
    assert dior == pytest.approx(J[0], rel=GRAD_RTOL, abs=1e-6 * max(1.0, abs(J[0])))
    np.testing.assert_allclose(dsig, J[1:], rtol=GRAD_RTOL, atol=1e-6 * max(1.0, np.abs(J[1:]).max()))


def test_ring_overflow_is_reported_and_retried(genus2):
    n0 = 2 * genus2.width * genus2.height * genus2.params.spp
    small = _checkpointed(genus2, level_capacity=n0 // 8)
    ws = dt.Workspace(dt.default_capacity(n0, 8), genus2.V.device, level_capacity=n0 // 8)
    _, tape = small.render(ws=ws, check=False)
    st = dt.read_stats(tape.ws)
    assert st["status"] == dt.DT_ERR_QUEUE_OVERFLOW and st["level_needed"] > n0 // 8
    img_c, tape_c = small.render()
    assert tape_c.ws.level_capacity >= tape_c.stats["level_needed"]
    img_f, _ = genus2.render()
    np.testing.assert_allclose(img_c.cpu().numpy(), img_f.cpu().numpy(), rtol=1e-6, atol=1e-7)


def test_checkpointed_batch_equals_full_batch(genus2):
    sc = S.glass_icosphere_scene(width=32, height=32)
    ico = GpuScene(sc.V, sc.F, 1.5, np.array([0.4, 0.2, 0.1], np.float32), sc.env, sc.cams, 32, 32, 5)
    full = [genus2, ico]
    ck = [_checkpointed(g) for g in full]

    def items(gl):
        return [dt.BatchItem(g.V, g.F, g.bvh, g.N, g.ior, g.sigma, g.env, g.cams, g.width, g.height, g.params)
                for g in gl]

    rng = np.random.default_rng(33)
    grads = [torch.from_numpy(rng.normal(size=(g.cams.shape[0], g.height, g.width, 3)).astype(np.float32)).cuda()
             for g in full]
    imgs_f, tape_f = dt.render_batch(items(full))
    out_f = dt.render_batch_backward(tape_f, grads)
    imgs_c, tape_c = dt.render_batch(items(ck))
    out_c = dt.render_batch_backward(tape_c, grads)
    assert tape_c.stats["segments"] == tape_f.stats["segments"]
    for a, b in zip(imgs_f, imgs_c):
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-6, atol=1e-7)
    for (dVa, dia, dsa), (dVb, dib, dsb) in zip(out_f, out_c):
        a, b = dVa.cpu().numpy().astype(np.float64), dVb.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(a), 1e-12)
        assert float(dib) == pytest.approx(float(dia), rel=1e-4, abs=1e-7)
    with pytest.raises(ValueError):
        dt.render_batch(items([full[0], ck[1]]))
