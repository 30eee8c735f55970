"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
closed-form eigenpairs, brute-force definitions on tiny grids, invariants,
exact solutions, and the paper's printed orders.  A plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import cgl_oracle as O
from paper_2403_02816_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers

def prob(n, bc, lo=-10.0, hi=10.0, **kw):
    d = len(n)
    par = dict(a1=1.0, b1=0.5, a2=1.0, a3=-1.0, b3=1.2, a4=0.0, b4=0.0)
    par.update(kw)
    return O.OracleProblem(tuple(n), tuple(bc), (lo,) * d, (hi,) * d, **par)


def rand_field(rng, n, scale=1.0):
    return scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n))


# ------------------------------------------------ FD matrices (closed form)

@pytest.mark.parametrize("n", [1, 2, 3, 7, 16])
def test_fd_dirichlet_eigenpairs(n):
    """tridiag(1,-2,1)/h^2 has eigenvalues -(4/h^2) sin^2(k pi/(2(n+1))) with
    eigenvectors sin(j k pi/(n+1)), j,k = 1..n."""
    lo, hi = -3.0, 5.0
    L = O.fd_laplacian(n, lo, hi, O.DIRICHLET)
    h = (hi - lo) / (n + 1)
    j = np.arange(1, n + 1)
    for k in range(1, n + 1):
        v = np.sin(j * k * np.pi / (n + 1))
        lam = -(4.0 / h**2) * np.sin(k * np.pi / (2 * (n + 1))) ** 2
        np.testing.assert_allclose(L @ v, lam * v, rtol=0, atol=1e-12 * abs(lam) * n)


@pytest.mark.parametrize("n", [2, 3, 8, 17])
def test_fd_neumann_eigenpairs(n):
    """Ghost-reflection Neumann matrix: eigenvalues -(4/h^2) sin^2(k pi/(2(n-1)))
    with eigenvectors cos(j k pi/(n-1)), j,k = 0..n-1."""
    lo, hi = -10.0, 10.0
    L = O.fd_laplacian(n, lo, hi, O.NEUMANN)
    h = (hi - lo) / (n - 1)
    j = np.arange(n)
    for k in range(n):
        v = np.cos(j * k * np.pi / (n - 1))
        lam = -(4.0 / h**2) * np.sin(k * np.pi / (2 * (n - 1))) ** 2
        np.testing.assert_allclose(L @ v, lam * v, rtol=0, atol=1e-12 * (4 / h**2) * n)


def _poly_d2(coef, x):
    import numpy.polynomial.polynomial as P
    return P.polyval(x, coef), P.polyval(x, P.polyder(coef, 2))


@pytest.mark.parametrize("deg", [2, 3, 4, 5])
def test_fd4_dirichlet_exact_on_quintics(deg):
    """The 4th-order Dirichlet matrix (Sec. 4.1.1) differentiates every
    polynomial of degree <= 5 that vanishes at both ends exactly (centred and
    one-sided rows alike), and no longer does so at degree 6."""
    import numpy.polynomial.polynomial as P
    lo, hi, n = -1.5, 2.0, 23
    h = (hi - lo) / (n + 1)
    x = lo + h * np.arange(1, n + 1)
    A = O.fd4_laplacian(n, lo, hi, O.DIRICHLET)
    for extra in (deg - 2, deg - 2 + 4):
        coef = P.polymul(P.polymul([-lo, 1.0], [hi, -1.0]), [0.3] * extra + [1.0])
        p, d2 = _poly_d2(coef, x)
        err = np.abs(A @ p - d2).max() / np.abs(d2).max()
        if extra + 2 <= 5:
            assert err < 1e-12, err
        else:
            assert err > 1e-6, err


@pytest.mark.parametrize("deg", [2, 3, 4])
def test_fd4_dirichlet_neumann_exact_on_quartics(deg):
    """The 4th-order mixed matrix (Sec. 4.2: Dirichlet at lo, Neumann at hi,
    semi-internal nodes) differentiates every polynomial of degree <= 4 with
    p(lo) = 0 and p'(hi) = 0 exactly, its two modified last rows included."""
    import numpy.polynomial.polynomial as P
    lo, hi, n = 0.5, 3.0, 19
    h = (hi - lo) / n
    x = lo + h * np.arange(1, n + 1)
    A = O.fd4_laplacian(n, lo, hi, O.NEUMANN)
    k = deg - 1
    base = [0.0] * k + [1.0] + [0.0] * 0  # x^k
    # p = (x - lo)(x^k + c), c chosen so that p'(hi) = 0
    c = -(hi ** k + (hi - lo) * k * hi ** (k - 1))
    q = list(base)
    q[0] += c
    coef = P.polymul([-lo, 1.0], q)
    p, d2 = _poly_d2(coef, x)
    assert abs(P.polyval(hi, P.polyder(coef, 1))) < 1e-12
    assert np.abs(A @ p - d2).max() / np.abs(d2).max() < 1e-12


def test_fd4_direction_matrices_override():
    """A problem carrying its own direction matrices uses them as given."""
    A = [O.fd4_laplacian(8, 0.0, 1.0, O.DIRICHLET) * complex(0.7, 0.2) + 0.1 * np.eye(8),
         O.fd4_laplacian(7, 0.0, 2.0, O.NEUMANN) * complex(0.7, 0.2) + 0.1 * np.eye(7)]
    p = O.OracleProblem((8, 7), (O.DIRICHLET, O.NEUMANN), (0.0, 0.0), (1.0, 2.0), 1.0, 0.0, 0.0, -1.0, 0.5,
                        mats=tuple(A))
    for mu in range(2):
        np.testing.assert_array_equal(O.direction_matrix(p, mu), A[mu])
    L = O.LinearOperator(p, 0.05)
    U = np.arange(56, dtype=complex).reshape(8, 7) / 56
    dense = O.expm(0.05 * O.kron_sum_dense(A)) @ O.to_vec(U)
    np.testing.assert_allclose(O.to_vec(L.expK(U, 1.0)), dense, atol=1e-13)


def test_fd_row_sums():
    """Neumann rows sum to zero (constants are in the kernel); Dirichlet
    first/last rows lose one neighbour."""
    L = O.fd_laplacian(9, 0.0, 1.0, O.NEUMANN)
    np.testing.assert_allclose(L.sum(axis=1), 0.0, atol=1e-9)
    D = O.fd_laplacian(9, 0.0, 1.0, O.DIRICHLET)
    h = 1.0 / 10
    assert D[0].sum() * h * h == pytest.approx(-1.0)
    assert D[4].sum() == pytest.approx(0.0, abs=1e-9)


# ------------------------------------------- small exponentials (spectral)

@pytest.mark.parametrize("bc,n", [(O.DIRICHLET, 12), (O.NEUMANN, 12), (O.DIRICHLET, 64),
                                  (O.NEUMANN, 33)])
@pytest.mark.parametrize("c", [1.0, 0.5])
def test_expm_matches_spectral_closed_form(bc, n, c):
    """exp(c tau A_mu) = S diag(exp(c tau ((a1+ib1) lam_k + a2/d))) S^{-1}
    with the closed-form sine/cosine eigenvectors S."""
    p = prob((n, n), (bc, bc))
    tau = 0.01
    A = O.direction_matrix(p, 0)
    lo, hi = p.lo[0], p.hi[0]
    if bc == O.DIRICHLET:
        h = (hi - lo) / (n + 1)
        j = np.arange(1, n + 1)
        ks = np.arange(1, n + 1)
        S = np.sin(np.outer(j, ks) * np.pi / (n + 1))
        lam = -(4.0 / h**2) * np.sin(ks * np.pi / (2 * (n + 1))) ** 2
    else:
        h = (hi - lo) / (n - 1)
        j = np.arange(n)
        ks = np.arange(n)
        S = np.cos(np.outer(j, ks) * np.pi / (n - 1))
        lam = -(4.0 / h**2) * np.sin(ks * np.pi / (2 * (n - 1))) ** 2
    mu = c * tau * (complex(p.a1, p.b1) * lam + p.a2 / p.d)
    ref = S @ np.diag(np.exp(mu)) @ np.linalg.inv(S)
    got = O.expm(c * tau * A)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_direction_matrix_splits_alpha2():
    """A_mu carries alpha2/d (the Kronecker sum then carries alpha2 once)."""
    p = prob((5, 5, 5), (O.DIRICHLET,) * 3, a2=0.9)
    A = O.direction_matrix(p, 1)
    L = O.fd_laplacian(5, -10, 10, O.DIRICHLET)
    np.testing.assert_allclose(A - complex(1.0, 0.5) * L, 0.3 * np.eye(5), atol=1e-14)


# -------------------------------------- Kronecker sum and Tucker (brute force)

def kron_sum_by_definition(mats):
    """K[(i),(j)] = sum_mu A_mu[i_mu, j_mu] prod_{nu != mu} delta(i_nu, j_nu),
    with the linear index i_1 + n_1 i_2 + n_1 n_2 i_3 (vec order)."""
    sizes = [M.shape[0] for M in mats]
    N = int(np.prod(sizes))
    K = np.zeros((N, N), dtype=complex)
    idx = list(np.ndindex(*reversed(sizes)))  # i_d slowest
    for a, ia in enumerate(idx):
        ia = ia[::-1]
        for b, ib in enumerate(idx):
            ib = ib[::-1]
            s = 0.0
            for mu in range(len(sizes)):
                if all(ia[nu] == ib[nu] for nu in range(len(sizes)) if nu != mu):
                    s += mats[mu][ia[mu], ib[mu]]
            K[a, b] = s
    return K


@pytest.mark.parametrize("n", [(3, 4), (2, 3, 2)])
def test_kron_sum_dense_matches_definition(n):
    rng = np.random.default_rng(1)
    mats = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for m in n]
    np.testing.assert_allclose(O.kron_sum_dense(mats), kron_sum_by_definition(mats), atol=1e-13)


@pytest.mark.parametrize("n,bc", [((8, 8), (O.DIRICHLET, O.DIRICHLET)),
                                  ((8, 5), (O.NEUMANN, O.DIRICHLET)),
                                  ((4, 4, 4), (O.DIRICHLET, O.NEUMANN, O.NEUMANN)),
                                  ((6,), (O.NEUMANN,))])
@pytest.mark.parametrize("c", [1.0, 0.5])
def test_tucker_equals_dense_expm(n, bc, c):
    """eq. Tucker: exp(c tau K) vec(U) = vec(U x_1 e^{c tau A_1} ... x_d e^{c tau A_d}),
    checked against expm of the assembled N x N Kronecker sum."""
    rng = np.random.default_rng(7)
    p = prob(n, bc)
    tau = 0.05
    L = O.LinearOperator(p, tau)
    U = rand_field(rng, n)
    K = kron_sum_by_definition(L.A)
    ref = O.from_vec(O.expm(c * tau * K) @ O.to_vec(U), n)
    got = L.expK(U, c)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_kronsumv_equals_dense():
    """eq. kronsumv: K u = vec(sum_mu U x_mu A_mu)."""
    rng = np.random.default_rng(3)
    p = prob((4, 3, 5), (O.NEUMANN, O.DIRICHLET, O.NEUMANN))
    L = O.LinearOperator(p, 0.1)
    U = rand_field(rng, p.n)
    K = kron_sum_by_definition(L.A)
    np.testing.assert_allclose(O.to_vec(L.K(U)), K @ O.to_vec(U), rtol=1e-12, atol=1e-10)


def test_mode_product_orientation():
    """(U x_mu M)_{..i..} = sum_j M[i,j] U_{..j..}: a non-square M on mode 2."""
    rng = np.random.default_rng(5)
    U = rng.standard_normal((2, 3, 4))
    M = rng.standard_normal((5, 3))
    V = O.mode_product(U, M, 1)
    assert V.shape == (2, 5, 4)
    for a in range(2):
        for i in range(5):
            for b in range(4):
                assert V[a, i, b] == pytest.approx(sum(M[i, j] * U[a, j, b] for j in range(3)))


# ------------------------------------------------- periodic (direct DFT)

def direct_dft(U, sign):
    """Non-separable O(N^2) DFT: sum_j U_j exp(sign 2 pi i sum_mu j_mu k_mu / n_mu)."""
    n = U.shape
    out = np.zeros(n, dtype=complex)
    for k in np.ndindex(*n):
        s = 0.0
        for j in np.ndindex(*n):
            ph = sum(j[m] * k[m] / n[m] for m in range(len(n)))
            s += U[j] * np.exp(sign * 2j * np.pi * ph)
        out[k] = s
    return out


@pytest.mark.parametrize("n", [(4, 6), (2, 4, 4)])
def test_periodic_linear_flow_matches_direct_dft(n):
    """E action (Sec. 3.2) = inverse DFT (1/N) of E times the forward DFT,
    with E from the signed wavenumbers; direct sums, no FFT."""
    rng = np.random.default_rng(11)
    p = prob(n, (O.PERIODIC,) * len(n), lo=-1.0, hi=2.0)
    tau = 0.02
    L = O.LinearOperator(p, tau)
    U = rand_field(rng, n)
    kap = [O.wavenumbers(n[m], p.lo[m], p.hi[m]) for m in range(len(n))]
    E = np.zeros(n, dtype=complex)
    for k in np.ndindex(*n):
        ksq = sum(kap[m][k[m]] ** 2 for m in range(len(n)))
        E[k] = np.exp(0.5 * tau * (complex(p.a1, p.b1) * (-ksq) + p.a2))
    N = int(np.prod(n))
    ref = direct_dft(E * direct_dft(U, -1), +1) / N
    np.testing.assert_allclose(L.expK(U, 0.5), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_periodic_single_mode_is_eigenfunction():
    """A lattice plane wave exp(i k.x) is multiplied by
    exp(c tau ((a1+ib1)(-|k|^2) + a2)) by the linear flow, and by
    (a1+ib1)(-|k|^2)+a2 by K; signed frequencies included."""
    p = prob((8, 16), (O.PERIODIC,) * 2, lo=-3.0, hi=5.0)
    P = I.Problem(p.n, p.bc, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3)
    for m in [(1, -3), (-4, 7), (3, 0)]:
        U = I.plane_wave_data(P, m, 1.0)
        k2 = sum((2 * np.pi * m[i] / (p.hi[i] - p.lo[i])) ** 2 for i in range(2))
        lam = complex(p.a1, p.b1) * (-k2) + p.a2
        L = O.LinearOperator(p, 0.03)
        np.testing.assert_allclose(L.expK(U, 1.0), np.exp(0.03 * lam) * U, atol=1e-13)
        np.testing.assert_allclose(L.K(U), lam * U, atol=1e-11)


# ------------------------------------------------ nonlinear flows

def fine_rk4(p, u, t, m=10000):
    h = t / m
    for _ in range(m):
        k1 = O.g(p, u)
        k2 = O.g(p, u + h / 2 * k1)
        k3 = O.g(p, u + h / 2 * k2)
        k4 = O.g(p, u + h * k3)
        u = u + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u


def test_g_definition():
    p = prob((1,), (O.PERIODIC,), a3=-0.7, b3=0.3, a4=-0.1, b4=0.2)
    u = np.array([0.3 - 0.8j])
    r = abs(u[0]) ** 2
    ref = (complex(-0.7, 0.3) * r + complex(-0.1, 0.2) * r * r) * u[0]
    assert O.g(p, u)[0] == pytest.approx(ref, rel=1e-15)


@pytest.mark.parametrize("a3,b3", [(-1.0, 1.2), (1.0, 1.0), (-2.0, -0.5), (0.0, 1.5)])
def test_phi_cubic_invariant_and_fine_rk4(a3, b3):
    """eq. exsolcub: |u(t)|^2 = |u0|^2 / (1 - 2 a3 |u0|^2 t); agrees with a
    1e4-substep RK4 integration of u' = (a3+ib3)|u|^2 u; a3 = 0 gives the pure
    phase rotation exp(i b3 |u0|^2 t)."""
    p = prob((1,), (O.PERIODIC,), a3=a3, b3=b3)
    rng = np.random.default_rng(2)
    u0 = rand_field(rng, (12,), 0.4)
    t = 0.3
    u = O.phi_cubic(p, u0, t)
    r0 = np.abs(u0) ** 2
    np.testing.assert_allclose(np.abs(u) ** 2, r0 / (1 - 2 * a3 * r0 * t), rtol=1e-13)
    np.testing.assert_allclose(u, fine_rk4(p, u0, t), rtol=1e-12, atol=1e-14)
    if a3 == 0.0:
        np.testing.assert_allclose(u, u0 * np.exp(1j * b3 * r0 * t), rtol=1e-14)


@pytest.mark.parametrize("a4,b4", [(-0.1, 0.1), (-1.0, -0.11), (0.0, 0.1)])
def test_phi_quintic_invariant_and_fine_rk4(a4, b4):
    """Sec. 4.3 quintic flow: |u|^4(t) = |u0|^4 / (1 - 4 a4 |u0|^4 t)."""
    p = prob((1,), (O.PERIODIC,), a3=0.0, b3=0.0, a4=a4, b4=b4)
    rng = np.random.default_rng(4)
    u0 = rand_field(rng, (10,), 0.6)
    t = 0.4
    u = O.phi_quintic(p, u0, t)
    r0 = np.abs(u0) ** 4
    np.testing.assert_allclose(np.abs(u) ** 4, r0 / (1 - 4 * a4 * r0 * t), rtol=1e-12)
    np.testing.assert_allclose(u, fine_rk4(p, u0, t), rtol=1e-12, atol=1e-14)


def test_rk4_nonlinear_local_order_five():
    """One RK4 step of u' = g(u) has local error O(t^5) against the exact
    cubic flow: halving t divides the error by ~32."""
    p = prob((1,), (O.PERIODIC,), a3=-1.0, b3=1.2)
    u0 = np.array([0.9 + 0.4j])
    e = [abs(O.rk4_nonlinear(p, u0, t) - O.phi_cubic(p, u0, t))[0] for t in (0.02, 0.01)]
    assert 28 < e[0] / e[1] < 36


def test_nonlinear_flow_selects_exact_or_rk4():
    u = np.array([0.5 + 0.5j])
    pc = prob((1,), (O.PERIODIC,))
    pq = prob((1,), (O.PERIODIC,), a4=-0.1, b4=0.1)
    assert O.nonlinear_flow(pc, u, 0.1)[0] == O.phi_cubic(pc, u, 0.1)[0]
    assert O.nonlinear_flow(pq, u, 0.1)[0] == O.rk4_nonlinear(pq, u, 0.1)[0]


# --------------------------------------------- schemes: exact plane waves

def plane_wave_problem(cubic):
    """Periodic 8x8 on (-pi, pi)^2; amplitude a and wave vector k fixed, a2
    chosen so that a exp(i(k.x - w t)) solves eq. (1) exactly:
    a2 - a1|k|^2 + a3 a^2 + a4 a^4 = 0,  w = b1|k|^2 - b3 a^2 - b4 a^4."""
    a, m = 0.8, (1, -2)
    a1, b1, a3, b3 = 0.6, 0.9, -0.8, 1.1
    a4, b4 = (0.0, 0.0) if cubic else (-0.3, 0.4)
    k2 = sum(v * v for v in m)
    a2 = a1 * k2 - a3 * a * a - a4 * a**4
    w = b1 * k2 - b3 * a * a - b4 * a**4
    p = O.OracleProblem((8, 8), (O.PERIODIC,) * 2, (-np.pi,) * 2, (np.pi,) * 2,
                        a1, b1, a2, a3, b3, a4, b4)
    P = I.Problem(p.n, p.bc, p.lo, p.hi, a1, b1, a2, a3, b3, a4, b4)
    U0 = I.plane_wave_data(P, m, a)
    return p, U0, w


def test_plane_wave_residual_vanishes():
    """The plane wave satisfies the semidiscrete ODE u' = K u + g(u) exactly."""
    for cubic in (True, False):
        p, U0, w = plane_wave_problem(cubic)
        L = O.LinearOperator(p, 0.1)
        np.testing.assert_allclose(L.K(U0) + O.g(p, U0), -1j * w * U0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2", "rk4", "rk2", "strang3t", "split4_3t"])
@pytest.mark.parametrize("cubic", [True, False])
def test_plane_wave_orders(scheme, cubic):
    """Temporal order on an exact solution (no spatial error): 2 for
    strang/lawson2/rk2, 4 for split4/lawson4/rk4, within +-0.1."""
    p, U0, w = plane_wave_problem(cubic)
    T = 1.0
    steps = (40, 80)
    errs = []
    for m in steps:
        U = O.integrate(p, U0, T / m, m, scheme)
        errs.append(O.rel_l2(U, U0 * np.exp(-1j * w * T)))
    order = O.observed_order(steps[0], errs[0], steps[1], errs[1])
    assert abs(order - O.ORDERS[scheme]) < 0.1, (errs, order)


# ---------------------------------- schemes: FD Neumann, spatially uniform

@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2", "rk4", "strang3t", "split4_3t"])
def test_neumann_uniform_solution_orders(scheme):
    """With Neumann conditions a constant field stays constant (the FD rows sum
    to zero) and solves u' = a2 u + (a3+ib3)|u|^2 u, whose closed form is
    u0 exp(a2 t + (a3+ib3) I(t)), I(t) = -log(1 - (a3/a2) r0 (e^{2 a2 t}-1))/(2 a3)."""
    p = prob((6, 5), (O.NEUMANN, O.NEUMANN), a2=0.7, a3=-1.3, b3=0.8)
    u0 = 0.6 - 0.3j
    U0 = np.full(p.n, u0, dtype=complex)
    T = 1.0
    r0 = abs(u0) ** 2
    It = -np.log(1 - (p.a3 / p.a2) * r0 * (np.exp(2 * p.a2 * T) - 1)) / (2 * p.a3)
    exact = u0 * np.exp(p.a2 * T + complex(p.a3, p.b3) * It)
    steps = (40, 80)
    errs = [O.rel_l2(O.integrate(p, U0, T / m, m, scheme), np.full(p.n, exact)) for m in steps]
    order = O.observed_order(steps[0], errs[0], steps[1], errs[1])
    assert abs(order - O.ORDERS[scheme]) < 0.1, (errs, order)


def test_three_term_splittings_reduce_to_two_term_for_cubic():
    """With a4 = b4 = 0 the quintic flow is the identity and the cubic flow is
    exact, so strang_3t is strang, and split4_3t is split4 (its two middle
    quarter flows compose to the half flow of split4's explicit form by the
    semigroup property of the exact flow) up to rounding."""
    p = O.OracleProblem((9, 6), (O.DIRICHLET, O.NEUMANN), (-3.0, -2.0), (3.0, 2.0), 0.8, 0.4, 0.5,
                        -1.1, 0.7, 0.0, 0.0)
    rng = np.random.default_rng(31)
    U0 = 0.5 * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
    for a, b in (("strang3t", "strang"), ("split4_3t", "split4")):
        ua = O.integrate(p, U0, 0.03, 5, a)
        ub = O.integrate(p, U0, 0.03, 5, b)
        assert O.rel_l2(ua, ub) < 1e-13, (a, O.rel_l2(ua, ub))


def test_three_term_nonlinear_parts_do_not_commute():
    """The cubic and quintic flows do not commute (already their radial parts
    r' = 2 a3 r^2 and r' = 2 a4 r^3 have the nonzero commutator 4 a3 a4 r^4),
    so the ordering inside strang_3t matters: phi^c o phi^q and phi^q o phi^c
    differ by O(t^2), a difference that quarters when t halves."""
    p = O.OracleProblem((4,), (O.PERIODIC,), (0.0,), (1.0,), 1.0, 0.0, 0.0, -0.9, 1.3, -0.4, 0.6)
    u = np.array([0.9 + 0.2j, -0.5 + 0.6j, 0.3 - 0.8j, 1.1 + 0.0j])
    d = []
    for t in (0.002, 0.001):
        cq = O.phi_cubic(p, O.phi_quintic(p, u, t), t)
        qc = O.phi_quintic(p, O.phi_cubic(p, u, t), t)
        d.append(np.abs(cq - qc).max())
    assert d[0] > 1e-6
    assert abs(np.log2(d[0] / d[1]) - 2.0) < 0.1


@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2", "strang3t", "split4_3t"])
def test_linear_problem_is_integrated_exactly(scheme):
    """With g = 0 every exponential scheme reproduces exp(tK) u0; a product of
    sine eigenvectors (Dirichlet) and cosine eigenvectors (Neumann) then
    evolves by exp(t sum_mu ((a1+ib1) lam_mu + a2/d))."""
    p = prob((9, 7), (O.DIRICHLET, O.NEUMANN), a3=0.0, b3=0.0)
    n1, n2 = p.n
    h1 = 20.0 / (n1 + 1)
    h2 = 20.0 / (n2 - 1)
    k1, k2 = 3, 2
    v1 = np.sin(np.arange(1, n1 + 1) * k1 * np.pi / (n1 + 1))
    v2 = np.cos(np.arange(n2) * k2 * np.pi / (n2 - 1))
    lam = (-(4 / h1**2) * np.sin(k1 * np.pi / (2 * (n1 + 1))) ** 2
           - (4 / h2**2) * np.sin(k2 * np.pi / (2 * (n2 - 1))) ** 2)
    U0 = np.outer(v1, v2).astype(complex)
    T, m = 0.3, 7
    U = O.integrate(p, U0, T / m, m, scheme)
    ref = np.exp(T * (complex(p.a1, p.b1) * lam + p.a2)) * U0
    np.testing.assert_allclose(U, ref, atol=1e-12 * np.abs(ref).max())


# --------------------------------------------- paper's printed orders

def test_observed_order_reproduces_paper_tables():
    """The order formula reproduces the orders printed in the paper's
    tables from the errors printed beside them."""
    rows = []
    with open(os.path.join(GOLDEN, "paper_orders.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) >= 8
    for tab, scheme, sa, ea, sb, eb, printed in rows:
        got = O.observed_order(int(sa), float(ea), int(sb), float(eb))
        assert abs(got - float(printed)) < 1e-2, (tab, scheme, got, printed)


# --------------------------------------------- error measures

def test_error_measures():
    ref = np.array([3.0, 4.0, 0.0])
    x = np.array([3.0, 4.0, 1.0])
    assert O.rel_l2(x, ref) == pytest.approx(1.0 / 5.0)
    assert O.rel_inf(x, ref) == pytest.approx(1.0 / 4.0)
