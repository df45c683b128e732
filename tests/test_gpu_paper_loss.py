"""The tracer stage's losses fused into the backward seed (Eq. 14: GT-weighted
L2; Eq. 15: tone, per pixel, averaged) against the FP64 oracle: values and
the image gradient, zero colours, an empty image, and the seed driving a
backward pass (dJ/dsigma through the renderer against the oracle's
forward-mode derivative chained with the oracle's loss gradient)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, PROBE, GpuScene, excluded_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def test_paper_losses_match_oracle():
    rng = np.random.default_rng(71)
    img = rng.uniform(0.0, 1.5, size=(3, 37, 29, 3)).astype(np.float32)
    tgt = rng.uniform(0.0, 1.0, size=img.shape).astype(np.float32)
    img[0, 0, :5] = 0.0  # rendered black: no cosine
    tgt[1, 2, :4] = 0.0  # true black
    g, loss = dt.paper_loss_grad(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), 0.6, 1.4)
    total, lc, lt, gref = O.paper_losses(img.astype(np.float64), tgt.astype(np.float64), 0.6, 1.4)
    np.testing.assert_allclose(loss.cpu().numpy(), [total, lc, lt], rtol=2e-5)
    # each gradient entry adds the colour and tone terms, which can cancel:
    # FP32 rounding is relative to the terms, so the floor is a small
    # fraction of the largest entry
    np.testing.assert_allclose(g.cpu().numpy(), gref, rtol=2e-5, atol=1e-6 * np.abs(gref).max())
    e, l0 = dt.paper_loss_grad(torch.zeros(0, 3, device="cuda"), torch.zeros(0, 3, device="cuda"))
    assert e.numel() == 0 and l0.cpu().numpy().tolist() == [0.0, 0.0, 0.0]


def test_paper_loss_seeds_the_backward():
    V, F = S.icosphere(3, 1.0)
    gs = GpuScene(V, F, 1.5, np.array([0.3, 0.1, 0.6], np.float32), S.sh_env_map(64, 32, 4),
                  S.fibonacci_views(1, 3.0, 24, 20), 24, 20, 4)
    p = gs.params
    orc = O.render(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, p.spp, p.jitter, p.seed,
                   0, p.t_min, probe=PROBE)
    img, tape = gs.render()
    # the true image: the render with another sigma, equal to ours on the
    # excluded pixels (so they seed nothing)
    tgt = O.render(gs.Vn, gs.Fn, gs.iorf, np.array([0.5, 0.2, 0.3]), gs.envn, gs.cam_list[0], p.max_depth)["img"]
    bad = excluded_pixels(orc, 0.0083)
    tgt[bad] = img[0].cpu().numpy()[bad]
    tgt32 = tgt.astype(np.float32)[None]
    seed, _ = dt.paper_loss_grad(img, torch.from_numpy(tgt32).cuda(), 1.0, 0.5)
    dsig = dt.render_backward(tape, seed)[2].cpu().numpy()
    tsig = np.eye(3)
    I, dI = O.render_jvp(gs.Vn, gs.Fn, gs.iorf, gs.sigman, gs.envn, gs.cam_list[0], p.max_depth, None, None, tsig)
    _, _, _, gref = O.paper_losses(img.cpu().numpy().astype(np.float64)[0], tgt32[0].astype(np.float64), 1.0, 0.5)
    gref[bad] = 0.0
    J = np.einsum("khwc,hwc->k", dI, gref)
    np.testing.assert_allclose(dsig, J, rtol=GRAD_RTOL, atol=1e-6 * max(1e-3, np.abs(J).max()))
