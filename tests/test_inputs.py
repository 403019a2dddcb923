"""Host logic of the seeded input generators shared by both sides of the parity tests (CPU)."""
import itertools

import numpy as np
import pytest

from paper_2602_05017_gb300 import inputs


def _on_face(v, nx, ny, nz):
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    return x in (0, nx - 1) or y in (0, ny - 1) or z in (0, nz - 1)


def test_face_value_nodes_cover_each_face_once_in_face_order():
    for nx, ny, nz in itertools.product([1, 2, 5], [1, 3, 4], [1, 2, 6]):
        faces = np.full((6, 2), np.nan)
        faces[:, 0] = np.arange(6) + 1.0          # substrate 0: all six faces
        faces[3, 1] = 9.0                         # substrate 1: the y+ face only
        vox, sub, val = inputs.face_value_nodes(nx, ny, nz, faces)
        assert vox.size == sub.size == val.size
        face_vox = {v for v in range(nx * ny * nz) if _on_face(v, nx, ny, nz)}
        s0 = vox[sub == 0]
        assert set(s0.tolist()) == face_vox
        # the value that stays at each voxel is the last listed one: the highest face index
        # among the faces it lies on (x-, x+, y-, y+, z-, z+)
        last = {}
        for v, s, x in zip(vox, sub, val):
            if s == 0:
                last[int(v)] = x
        for v in face_vox:
            x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
            on = [x == 0, x == nx - 1, y == 0, y == ny - 1, z == 0, z == nz - 1]
            assert last[v] == max(f for f in range(6) if on[f]) + 1.0
        s1 = vox[sub == 1]
        assert set(s1.tolist()) == {v for v in range(nx * ny * nz) if (v // nx) % ny == ny - 1}
        assert np.all(val[sub == 1] == 9.0)


def test_random_nodes_are_seeded_in_range_and_repeat_some_pairs():
    a = inputs.random_nodes(np.random.default_rng(5), 1000, 3, 40)
    b = inputs.random_nodes(np.random.default_rng(5), 1000, 3, 40)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    vox, sub, val = a
    assert vox.min() >= 0 and vox.max() < 1000 and sub.min() >= 0 and sub.max() < 3
    assert np.all((val >= 0) & (val <= 38))
    k = 40 // 8
    np.testing.assert_array_equal(vox[-k:], vox[:k])
    np.testing.assert_array_equal(sub[-k:], sub[:k])


def test_random_problem_draws_are_unchanged_by_the_node_option():
    """Adding Dirichlet nodes draws after everything else: the rest of a seeded problem is the
    same with and without them."""
    p = inputs.random_problem(np.random.default_rng(8), 6, 5, 4, 2, n_agents=7, dirichlet=True)
    q = inputs.random_problem(np.random.default_rng(8), 6, 5, 4, 2, n_agents=7, dirichlet=True,
                              n_nodes=9)
    np.testing.assert_array_equal(p.rho0, q.rho0)
    np.testing.assert_array_equal(p.voxel, q.voxel)
    assert p.dirichlet_nodes is None and len(q.dirichlet_nodes[0]) == 9


def test_blob_field_draws_do_not_depend_on_with_field():
    """Workload 3 draws its blob parameters before its agents whether or not the host field is
    formed, so a device-evaluated field pairs with the same agents."""
    a = inputs.workload(3, shape=(20, 18, 16), n_agents=50)
    b = inputs.workload(3, shape=(20, 18, 16), n_agents=50, with_field=False)
    np.testing.assert_array_equal(a.voxel, b.voxel)
    np.testing.assert_array_equal(a.secretion, b.secretion)
    for x, y in zip(a.extra["blobs"], b.extra["blobs"]):
        np.testing.assert_array_equal(x, y)
    assert b.rho0 is None and a.rho0.shape == (16, 18, 20, 2) and a.rho0.max() > 0


def test_device_blob_evaluator_matches_the_host_one_on_cpu():
    import torch
    w = inputs.workload(3, shape=(24, 20, 18), n_agents=10)
    got = inputs.gaussian_blobs_device(w.extra["blobs"], w.nx, w.ny, w.nz, 2, w.dx, "cpu")
    np.testing.assert_allclose(got.numpy(), w.rho0, rtol=1e-13, atol=1e-12 * w.rho0.max())
    assert got.dtype == torch.float64


def test_first_substrates_keeps_the_leading_columns():
    w = inputs.workload(2, shape=(8, 6, 5), n_agents=12)
    v = inputs.first_substrates(w, 2)
    assert v.ns == 2 and v.rho0.shape == (5, 6, 8, 2)
    assert np.array_equal(v.rho0, w.rho0[..., :2]) and np.array_equal(v.D, w.D[:2])
    assert np.array_equal(v.secretion, w.secretion[:, :2]) and np.array_equal(v.voxel, w.voxel)
    with pytest.raises(ValueError):
        inputs.first_substrates(w, 5)
