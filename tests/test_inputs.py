"""Seeded workload generators: determinism, shapes and node conventions."""
import numpy as np

from paper_2403_02816_gb300 import inputs as I


def test_seeded_fields_are_reproducible():
    w = I.workload_2d_dirichlet(16)
    a = I.u0_2d_dirichlet(w)
    b = I.u0_2d_dirichlet(w)
    assert a.shape == (16, 16) and a.dtype == np.complex128
    np.testing.assert_array_equal(a, b)


def test_node_conventions():
    np.testing.assert_allclose(I.nodes(3, 0.0, 4.0, I.DIRICHLET), [1.0, 2.0, 3.0])
    np.testing.assert_allclose(I.nodes(3, 0.0, 4.0, I.NEUMANN), [0.0, 2.0, 4.0])
    np.testing.assert_allclose(I.nodes(4, 0.0, 4.0, I.PERIODIC), [0.0, 1.0, 2.0, 3.0])


def test_device_layout_is_vec_order():
    U = np.arange(6).reshape(2, 3).astype(complex)
    np.testing.assert_array_equal(I.device_layout(U), [0, 3, 1, 4, 2, 5])
    np.testing.assert_array_equal(I.from_device_layout(I.device_layout(U), (2, 3)), U)


def test_smooth_field_rms():
    w = I.workload_3d_neumann(16)
    U = I.u0_3d_neumann(w)
    assert abs(np.sqrt(np.mean(np.abs(U) ** 2)) - 0.1) < 1e-12


def test_batched_problem_ranges():
    ps = I.batched_problems(64)
    assert len(ps) == 64
    for p in ps:
        assert all(48 <= n <= 256 for n in p.n)
        assert all(b in (I.DIRICHLET, I.NEUMANN) for b in p.bc)
        assert 0.2 <= p.a1 <= 2 and -2 <= p.a3 <= -0.5 and p.a4 in (0.0, -0.1)
