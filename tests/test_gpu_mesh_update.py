"""The step after the gradient (App. A) on the device against the FP64
oracle (oracle/mesh_update.py): the mesh's edge graph, the large-steps
solve (I + lambda L) x = b, the AdamUniform update over several steps, a
constant gradient translating the mesh, and L_edge with its vertex
gradient."""
import numpy as np
import pytest
import torch

import paper_2603_00413_gb300 as dt
from oracle import mesh_update as MU
from paper_2603_00413_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2603_00413_gb300 import build
    build.build()


def _meshes():
    yield "icosphere3", S.icosphere(3)
    yield "tori", S.two_tori_mesh(24)
    V, F = S.icosphere(1)
    # a repeated face and a face with a repeated vertex: no extra edges
    F2 = np.concatenate([F, F[:1], np.array([[0, 0, 1]], np.int32)])
    yield "odd", (V, F2)


@pytest.mark.parametrize("name,mesh", list(_meshes()), ids=lambda x: x if isinstance(x, str) else "")
def test_topology_is_the_edge_graph(name, mesh):
    V, F = mesh
    topo = dt.Topology(torch.from_numpy(np.asarray(F, np.int32)).cuda(), len(V))
    ne, md, row, col = topo.info()
    row, col = row.cpu().numpy(), col.cpu().numpy()
    E = MU.edges(F)
    assert ne == len(E)
    got = np.array([(i, j) for i in range(len(V)) for j in col[row[i]:row[i + 1]] if j > i])
    np.testing.assert_array_equal(got, E)
    deg = np.diff(row)
    assert md == deg.max()
    np.testing.assert_array_equal(deg, MU.laplacian(F, len(V)).diagonal())


def test_smooth_solve_matches_oracle():
    V, F = S.two_tori_mesh(24)
    rng = np.random.default_rng(91)
    b = rng.normal(size=(len(V), 3))
    topo = dt.Topology(torch.from_numpy(F).cuda(), len(V))
    x = dt.smooth_solve(topo, 10.0, torch.from_numpy(b.astype(np.float32)).cuda(), iters=300)
    ref = MU.smooth_solve(F, len(V), 10.0, b)
    # the solve stops once a column's residual has fallen by 1e-6; the
    # error is then bounded by that times the square root of the
    # preconditioned condition number (about 2 (1 + lambda deg) here)
    err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-6 * np.sqrt(2 * (1 + 10.0 * 8)) * 4, err


def test_large_steps_updates_match_oracle():
    V, F = S.icosphere(3)
    rng = np.random.default_rng(92)
    Vd = V.astype(np.float64)
    Vg = torch.from_numpy(V.copy()).cuda()
    opt = dt.LargeStepsOptimizer(Vg, torch.from_numpy(F).cuda(), lam=8.0, lr=0.02, iters=300)
    st = None
    for _ in range(3):
        g = rng.normal(size=V.shape)
        opt.step(torch.from_numpy(g.astype(np.float32)).cuda())
        Vd, st = MU.large_steps_update(F, Vd, g.astype(np.float32).astype(np.float64), st, lam=8.0, lr=0.02)
    got = Vg.cpu().numpy()
    assert np.abs(got - Vd).max() <= 1e-4 * np.abs(Vd).max()
    assert np.abs(got - V).max() > 1e-3  # it moved


def test_large_steps_constant_gradient_translates():
    V, F = S.icosphere(2)
    Vg = torch.from_numpy(V.copy()).cuda()
    opt = dt.LargeStepsOptimizer(Vg, torch.from_numpy(F).cuda(), lam=12.0, lr=0.01, iters=200)
    c = np.array([0.5, -2.0, 1.0], np.float32)
    opt.step(torch.from_numpy(np.tile(c, (len(V), 1))).cuda())
    np.testing.assert_allclose(Vg.cpu().numpy(), V - 0.01 * c / 2.0, rtol=0, atol=2e-6)


def test_edge_loss_matches_oracle():
    V, F = S.icosphere(3)
    rng = np.random.default_rng(93)
    V = (V * (1.0 + 0.05 * rng.uniform(size=(len(V), 1)))).astype(np.float32)
    loss, dV = dt.edge_loss_grad(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
    ref_loss, ref_dV = MU.edge_loss(V.astype(np.float64), F)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-4)
    got = dV.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref_dV) <= 1e-4 * np.linalg.norm(ref_dV)
