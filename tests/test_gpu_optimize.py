"""The optimisation loop of the tracer stage end to end on the device: render,
the paper's colour and tone losses as the seed (Eqs. 14-15), the backward,
L_edge's gradient added, the large-steps update of the mesh with AdamUniform
(App. A) and plain Adam steps on the IoR and sigma.  Starting from a
smoothly dented sphere with the wrong IoR and absorption, 40 steps must
halve the image loss and the material error and bring the vertex error
down."""
import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def test_optimisation_loop_recovers_shape_and_material():
    dev = torch.device("cuda:0")
    V0, F = S.icosphere(3)
    rng = np.random.default_rng(101)
    d = V0 / np.linalg.norm(V0, axis=1, keepdims=True)
    dent = 0.06 * np.tanh(3.0 * (d @ np.array([0.6, 0.8, 0.0])))  # a smooth dent across the sphere
    Vstart = (V0 * (1.0 + dent[:, None])).astype(np.float32)
    env = torch.from_numpy(S.sh_env_map(64, 32, 5)).to(dev)
    cams = torch.from_numpy(np.stack([c.as_array() for c in S.fibonacci_views(4, 3.0, 40, 40)])).to(dev)
    Ft = torch.from_numpy(F).to(dev)
    params = dt.Params(4)
    ior_true = torch.tensor([1.5], device=dev)
    sig_true = torch.tensor([0.3, 0.1, 0.2], device=dev)
    Vt = torch.from_numpy(V0).to(dev)
    target, _ = dt.render(Vt, Ft, dt.build_bvh(Vt, Ft), dt.vertex_normals(Vt, Ft), ior_true, sig_true, env, cams,
                          40, 40, params)
    V = torch.from_numpy(Vstart.copy()).to(dev)
    ior = torch.tensor([1.4], device=dev)
    sig = torch.tensor([0.6, 0.3, 0.05], device=dev)
    topo = dt.Topology(Ft, V.shape[0])
    opt_v = dt.LargeStepsOptimizer(V, Ft, lam=10.0, lr=5e-3, topo=topo)
    mat = torch.cat([ior, sig]).clone()
    m = torch.zeros_like(mat)
    v = torch.zeros_like(mat)
    bvh = dt.build_bvh(V, Ft)
    losses, verr, merr = [], [], []
    for it in range(40):
        bvh.refit(V, Ft)
        N = dt.vertex_normals(V, Ft)
        img, tape = dt.render(V, Ft, bvh, N, mat[:1].contiguous(), mat[1:].contiguous(), env, cams, 40, 40, params)
        seed, loss = dt.paper_loss_grad(img, target, 1.0, 0.1)
        dV, dior, dsig = dt.render_backward(tape, seed)
        le, dVe = dt.edge_loss_grad(V, Ft, topo)
        opt_v.step(dV + 1e-3 * dVe)
        g = torch.cat([dior, dsig])
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        mat -= 0.01 * (m / (1 - 0.9 ** (it + 1))) / (torch.sqrt(v / (1 - 0.999 ** (it + 1))) + 1e-8)
        mat[1:].clamp_(min=0.0)
        losses.append(float(loss[0]))
        verr.append(float((V - Vt).norm(dim=1).mean()))
        merr.append(float((mat - torch.cat([ior_true, sig_true])).abs().max()))
    assert losses[-1] < 0.5 * losses[0], losses[::8]
    assert verr[-1] < 0.95 * verr[0], verr[::8]  # geometry through refraction moves slowly
    assert merr[-1] < 0.5 * merr[0], merr[::8]
