"""The benchmark workload at full size, in the launch configuration bench.py
times: the genus-2 two-tori mesh (~52.5k triangles), 100 views at 512x512,
depth 8.  The oracle cannot render 26M pixels, so it checks a seeded sample
of them one by one (radiance), and the gradient of a loss seeded only on
those pixels (exact, by forward mode over every parameter they can touch)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S
from tests.gpu_util import GRAD_RTOL, PROBE, RAD_ATOL, RAD_RTOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_2603_00413_gb300 import build
    build.build()
    sc, _ = S.genus2_scene()
    dev = torch.device("cuda:0")
    V = torch.from_numpy(sc.V).to(dev)
    F = torch.from_numpy(sc.F).to(dev)
    ior = torch.tensor([sc.ior], device=dev)
    sigma = torch.from_numpy(sc.sigma).to(dev)
    env = torch.from_numpy(sc.env).to(dev)
    cams = torch.from_numpy(np.stack([c.as_array() for c in sc.cams])).to(dev)
    N = dt.vertex_normals(V, F)
    bvh = dt.build_bvh(V, F)
    params = dt.Params(sc.max_depth)
    img, tape = dt.render(V, F, bvh, N, ior, sigma, env, cams, 512, 512, params)
    return sc, img, tape


def _rays(sc, views, pix):
    o = np.zeros((len(views), 3))
    d = np.zeros((len(views), 3))
    for i, (v, p) in enumerate(zip(views, pix)):
        oo, dd = O.camera_rays(sc.cams[v])
        o[i], d[i] = oo[p], dd[p]
    return o, d


def _sample(sc, n, seed, hits_only=False):
    """n seeded (view, pixel) samples with their camera rays; with hits_only,
    drawn (in rounds of candidates) among pixels whose path hits the object
    and is not edge-degenerate."""
    rng = np.random.default_rng(seed)
    if not hits_only:
        views = rng.integers(0, len(sc.cams), size=n)
        pix = rng.integers(0, 512 * 512, size=n)
        o, d = _rays(sc, views, pix)
        return views, pix, o, d
    got_v, got_p = [], []
    for _ in range(12):
        m = 8 * n
        views = rng.integers(0, len(sc.cams), size=m)
        pix = rng.integers(0, 512 * 512, size=m)
        o, d = _rays(sc, views, pix)
        r = O.render_rays(sc.V, sc.F, sc.ior, sc.sigma, sc.env, o, d, sc.max_depth, probe=PROBE, segments=True)
        hit = np.zeros(m, bool)
        hit[np.unique(r["seg_i"][r["seg_i"][:, 2] >= 0, 0])] = True
        keep = np.nonzero(hit & ((r["pix_flags"] & O.SEG_DEGENERATE) == 0))[0]
        got_v += list(views[keep])
        got_p += list(pix[keep])
        if len(got_v) >= n:
            break
    assert len(got_v) >= n
    views, pix = np.array(got_v[:n]), np.array(got_p[:n])
    o, d = _rays(sc, views, pix)
    return views, pix, o, d


def test_full_size_forward_sampled_pixels(full):
    sc, img, tape = full
    st = tape.stats
    assert st["status"] == dt.DT_OK
    assert st["n_levels"] == sc.max_depth + 1
    assert st["level_count"][0] == 100 * 512 * 512
    views, pix, o, d = _sample(sc, 96, 5)
    r = O.render_rays(sc.V, sc.F, sc.ior, sc.sigma, sc.env, o, d, sc.max_depth, probe=PROBE)
    ok = (r["pix_flags"] & O.SEG_DEGENERATE) == 0
    assert ok.mean() > 0.6
    # and a sample among pixels that reach the object
    hv, hp, ho, hd = _sample(sc, 48, 8, hits_only=True)
    rh = O.render_rays(sc.V, sc.F, sc.ior, sc.sigma, sc.env, ho, hd, sc.max_depth)
    gh = img.view(100, -1, 3)[torch.from_numpy(hv).cuda(), torch.from_numpy(hp).cuda()].cpu().numpy()
    assert (np.abs(gh - rh["img"]) <= RAD_RTOL * np.abs(rh["img"]) + RAD_ATOL).all()
    g = img.view(100, -1, 3)[torch.from_numpy(views).cuda(), torch.from_numpy(pix).cuda()].cpu().numpy()
    err = np.abs(g - r["img"])
    assert (err[ok] <= RAD_RTOL * np.abs(r["img"][ok]) + RAD_ATOL).all(), err[ok].max()


def test_full_size_gradient_of_sampled_pixels(full):
    sc, img, tape = full
    views, pix, o, d = _sample(sc, 12, 6, hits_only=True)
    rng = np.random.default_rng(7)
    gs = rng.normal(size=(12, 3))
    grad = torch.zeros(100, 512 * 512, 3, device="cuda")
    grad[torch.from_numpy(views).cuda(), torch.from_numpy(pix).cuda()] = torch.from_numpy(gs.astype(np.float32)).cuda()
    dV, dior, dsig = dt.render_backward(tape, grad.view(100, 512, 512, 3))
    dVo, dioro, dsigo, _ = O.rays_grad(sc.V, sc.F, sc.ior, sc.sigma, sc.env, o, d, sc.max_depth, gs)
    assert float(dior) == pytest.approx(dioro, rel=GRAD_RTOL, abs=1e-6)
    np.testing.assert_allclose(dsig.cpu().numpy(), dsigo, rtol=GRAD_RTOL, atol=1e-6)
    dVg = dV.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(dVg - dVo) / np.linalg.norm(dVo)
    assert rel < GRAD_RTOL, rel
