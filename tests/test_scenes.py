"""The seeded input generators make what the workloads describe: closed,
outward-oriented meshes of the stated size and genus; smooth positive
environment maps; deterministic output per seed."""
import numpy as np
import pytest

from paper_2603_00413_gb300 import scenes as S


def test_icosphere_counts_and_closedness():
    for s, nv, nf in [(0, 12, 20), (1, 42, 80), (3, 642, 1280)]:
        V, F = S.icosphere(s)
        st = S.check_closed_mesh(V, F)
        assert (st["nv"], st["nf"], st["genus"]) == (nv, nf, 0)
        assert V.dtype == np.float32 and F.dtype == np.int32
        np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, rtol=1e-6)


def test_two_tori_is_genus_two_with_about_50k_faces():
    V, F = S.two_tori_mesh()
    st = S.check_closed_mesh(V, F)
    assert st["genus"] == 2
    assert 45000 <= st["nf"] <= 56000
    assert np.linalg.norm(V.astype(np.float64), axis=1).max() <= 1.0 + 1e-6


def test_random_blob_meshes_are_closed_and_sized():
    rng = np.random.default_rng(2)
    for target in (2000, 8000):
        V, F = S.mesh_from_field(S.random_blob_field(rng), target)
        st = S.check_closed_mesh(V, F)
        assert 0.8 * target <= st["nf"] <= 1.25 * target


def test_box_grid_closed():
    V, F = S.box_grid(3, (1.0, 1.0, 0.2))
    st = S.check_closed_mesh(V, F)
    assert st["genus"] == 0 and st["nf"] == 6 * 9 * 2
    assert abs(st["volume"] - 1.6) < 1e-6  # 2 x 2 x 0.4


def test_env_map_smooth_positive_deterministic():
    a = S.sh_env_map(64, 32, 0)
    b = S.sh_env_map(64, 32, 0)
    c = S.sh_env_map(64, 32, 1)
    assert a.shape == (32, 64, 3) and a.dtype == np.float32
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert (a > 0).all()
    # smooth: neighbouring texels differ by far less than the spread
    assert np.abs(np.diff(a, axis=1)).max() < 0.5 * (a.max() - a.min())


def test_real_sh_basis_is_orthonormal():
    """Quadrature of Y_lm Y_l'm' over the sphere on a fine grid = identity."""
    H, W = 200, 400
    TH, PH = S.texel_directions(W, H)
    Y = S._real_sh_basis(4, TH, PH)
    w = np.sin(TH) * (np.pi / H) * (2 * np.pi / W)
    G = np.einsum("khw,jhw,hw->kj", Y, Y, w)
    np.testing.assert_allclose(G, np.eye(25), atol=2e-3)


def test_fibonacci_views_on_sphere():
    cams = S.fibonacci_views(100, 3.0, 512, 512)
    E = np.array([c.eye for c in cams])
    np.testing.assert_allclose(np.linalg.norm(E, axis=1), 3.0, rtol=1e-6)
    assert abs(E.mean(axis=0)).max() < 0.1


def test_hash_texture_inputs():
    """Level sizes grow geometrically from n_min to n_max (Instant-NGP's level
    scale); the table is seeded, non-negative and averages the requested
    rate over the levels; the step defaults to half the finest cell."""
    assert S.hash_texture_resolutions(1, 16, 128) == [16]
    res = S.hash_texture_resolutions(8, 16, 128)
    assert res[0] == 16 and res[-1] == 128 and all(b > a for a, b in zip(res, res[1:]))
    ratios = np.array(res[1:], float) / np.array(res[:-1], float)
    assert np.allclose(ratios, 2 ** (3 / 7), atol=0.06)
    a = S.random_hash_texture(4, 10, 4, 32, (-1, -1, -1), (1, 1, 1), seed=3, scale=2.0)
    b = S.random_hash_texture(4, 10, 4, 32, (-1, -1, -1), (1, 1, 1), seed=3, scale=2.0)
    assert a["table"].shape == (4, 1024, 3) and a["table"].dtype == np.float32
    assert np.array_equal(a["table"], b["table"]) and a["res"] == b["res"] == [4, 8, 16, 32]
    assert a["table"].min() >= 0 and abs(a["table"].sum(axis=0).mean() - 2.0) < 0.1
    assert a["step"] == pytest.approx(0.5 * 2.0 / 31, rel=1e-6)
