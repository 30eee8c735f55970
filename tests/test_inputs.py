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


def test_coupled_workload_is_the_papers_grid_and_a_mirrored_soliton_pair():
    p = I.coupled_problem()
    assert p.n == (700, 350) and p.hi == (70.0, 35.0) and (p.a0, p.a5) == (-0.4, 0.5)
    W = I.coupled_u0(p)
    assert W.shape == (2, 700, 350) and W.dtype == np.complex128
    np.testing.assert_array_equal(W, I.coupled_u0(p))  # seeded
    x1 = I.nodes(700, 0.0, 70.0, I.PERIODIC)
    # u peaks at chi = 17.5, v at 70 - 17.5; amplitude delta = 2.25 up to the 1e-3 noise
    assert abs(x1[np.argmax(np.abs(W[0, :, 0]))] - 17.5) < 0.15
    assert abs(x1[np.argmax(np.abs(W[1, :, 0]))] - 52.5) < 0.15
    assert abs(np.max(np.abs(W[0])) - 2.25) < 0.02
    # without the noise v0(x1) = u0(70 - x1): the envelopes agree to the noise level
    mirror = np.roll(np.abs(W[0])[::-1, :], 1, axis=0)
    assert np.max(np.abs(mirror - np.abs(W[1]))) < 0.03
