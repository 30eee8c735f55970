"""Plain, slow FP64 CPU oracle for the exponential CGL integrators of
Caliari & Cassini, "Efficient simulation of complex Ginzburg-Landau equations
using high-order exponential-type methods" (arXiv 2403.02816).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs use it.  It shares no code with
the CUDA library and imports nothing from the package.

Everything is float64 / complex128 numpy.  Library primitives used as single
steps: ``numpy.tensordot`` (a matrix product), ``numpy.fft.fftn/ifftn`` (an
FFT) and ``scipy.linalg.expm`` (the Pade scaling-and-squaring matrix
exponential the paper itself uses, Sec. 4 "Numerical experiments").

Tensor convention.  A grid function is an array ``U`` of shape
``(n_1, ..., n_d)`` indexed like the paper's U_{i_1...i_d}; the paper's
``vec(U)`` (Sec. 3.1, stacking columns so that i_1 runs fastest) is
``U.reshape(-1, order="F")``.  Helpers ``to_vec``/``from_vec`` convert.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py``
against something other than itself (closed forms, brute force, invariants,
exact solutions, the paper's printed orders).  No function is parity-unpinned.

Readings of the paper where it is silent (2nd-order FD matrices, signed
Fourier wavenumbers, the stable form of the cubic flow, ...) are stated at
each function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Sequence

import numpy as np
import scipy.linalg

# --------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------

DIRICHLET, NEUMANN, PERIODIC = 0, 1, 2


@dataclass
class OracleProblem:
    """Eq. (1): u_t = (a1+i b1) Lap u + a2 u + (a3+i b3)|u|^2 u + (a4+i b4)|u|^4 u
    on Omega = (lo_1,hi_1) x ... x (lo_d,hi_d) with per-direction boundary
    conditions ``bc`` (DIRICHLET / NEUMANN / PERIODIC)."""

    n: tuple
    bc: tuple
    lo: tuple
    hi: tuple
    a1: float
    b1: float
    a2: float
    a3: float
    b3: float
    a4: float = 0.0
    b4: float = 0.0
    # optional caller-supplied direction matrices A_mu (complex n_mu x n_mu),
    # replacing (a1 + i b1) D2_mu + a2/d; e.g. the paper's 4th-order FD
    mats: tuple = None

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def periodic(self) -> bool:
        return all(b == PERIODIC for b in self.bc)

    @property
    def cubic(self) -> bool:
        """alpha4 = beta4 = 0: the cubic CGL (Sec. 1)."""
        return self.a4 == 0.0 and self.b4 == 0.0


def as_problem(p) -> OracleProblem:
    """Accept any object with the OracleProblem attributes (duck typing)."""
    if isinstance(p, OracleProblem):
        return p
    return OracleProblem(tuple(p.n), tuple(p.bc), tuple(p.lo), tuple(p.hi),
                         p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)


def to_vec(U: np.ndarray) -> np.ndarray:
    """vec(U): stack the columns, i_1 fastest (Sec. 3.1, eq. kronsumv)."""
    return U.reshape(-1, order="F")


def from_vec(u: np.ndarray, n: Sequence[int]) -> np.ndarray:
    return np.asarray(u).reshape(tuple(n), order="F")


# --------------------------------------------------------------------------
# Space discretisation (Sec. 1 eq. (2); Sec. 3.1 and 3.2)
# --------------------------------------------------------------------------

def fd_laplacian(n: int, lo: float, hi: float, bc: int) -> np.ndarray:
    """Second-order finite-difference d^2/dx^2 on one direction.

    The paper prints 4th-order matrices (Sec. 4.1.1, 4.2); the workloads use
    2nd order, so this is the reading adopted for it:
      * DIRICHLET: n interior nodes x_j = lo + j h, j = 1..n, h = (hi-lo)/(n+1),
        tridiag(1, -2, 1)/h^2.
      * NEUMANN: n nodes including both boundary nodes, x_j = lo + j h,
        j = 0..n-1, h = (hi-lo)/(n-1); a reflected ghost node gives first row
        (-2, 2)/h^2 and last row (2, -2)/h^2.
    """
    if bc == DIRICHLET:
        h = (hi - lo) / (n + 1)
    elif bc == NEUMANN:
        if n < 2:
            raise ValueError("Neumann needs n >= 2")
        h = (hi - lo) / (n - 1)
    else:
        raise ValueError("fd_laplacian: bc must be DIRICHLET or NEUMANN")
    L = np.zeros((n, n))
    for j in range(n):
        L[j, j] = -2.0
        if j > 0:
            L[j, j - 1] = 1.0
        if j < n - 1:
            L[j, j + 1] = 1.0
    if bc == NEUMANN and n >= 2:
        L[0, 1] = 2.0
        L[n - 1, n - 2] = 2.0
    return L / (h * h)


def fd4_laplacian(n: int, lo: float, hi: float, right: int = DIRICHLET) -> np.ndarray:
    """The paper's 4th-order finite-difference d^2/dx^2 matrices, as printed.

      * right = DIRICHLET (Sec. 4.1.1): homogeneous Dirichlet at both ends, n
        internal nodes x_j = lo + j h, j = 1..n, h = (hi-lo)/(n+1); centred
        rows (-1, 16, -30, 16, -1)/(12 h^2), and in the first and last rows
        the one-sided (-15, -4, 14, -6, 1)/(12 h^2) (the boundary value, zero,
        drops out) and its mirror image.
      * right = NEUMANN (Sec. 4.2, "semi-internal nodes"): Dirichlet at lo,
        homogeneous Neumann at hi, nodes x_j = lo + j h, j = 1..n, h =
        (hi-lo)/n (x_n = hi); first row as above, the last two rows
        (1, -6, 14, -4, -15, 10)/(12 h^2) and (1, -8/3, -6, 56, -145/3)/(12 h^2)
        on the last six and five nodes.
    """
    if n < 6:
        raise ValueError("fd4_laplacian needs n >= 6")
    if right == DIRICHLET:
        h = (hi - lo) / (n + 1)
    elif right == NEUMANN:
        h = (hi - lo) / n
    else:
        raise ValueError("fd4_laplacian: right must be DIRICHLET or NEUMANN")
    A = np.zeros((n, n))
    for i in range(n):
        for off, c in zip(range(-2, 3), (-1.0, 16.0, -30.0, 16.0, -1.0)):
            if 0 <= i + off < n:
                A[i, i + off] = c
    A[0, :] = 0.0
    A[0, :5] = [-15.0, -4.0, 14.0, -6.0, 1.0]
    if right == DIRICHLET:
        A[n - 1, :] = 0.0
        A[n - 1, n - 5:] = [1.0, -6.0, 14.0, -4.0, -15.0]
    else:
        A[n - 2, :] = 0.0
        A[n - 2, n - 6:] = [1.0, -6.0, 14.0, -4.0, -15.0, 10.0]
        A[n - 1, :] = 0.0
        A[n - 1, n - 5:] = [1.0, -8.0 / 3.0, -6.0, 56.0, -145.0 / 3.0]
    return A / (12.0 * h * h)


def wavenumbers(n: int, lo: float, hi: float) -> np.ndarray:
    """Signed Fourier wavenumbers kappa_m = 2 pi m / (hi - lo) in FFT order
    m = 0..n/2-1, -n/2..-1.  Sec. 3.2 writes (j-1)^2 on (0, 2 pi); the signed
    reading is the one for which the pseudospectral method is consistent (only
    kappa^2 enters, so the sign of the Nyquist mode does not matter)."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return 2.0 * np.pi * m / (hi - lo)


def direction_matrix(p: OracleProblem, mu: int) -> np.ndarray:
    """A_mu ~ (a1 + i b1) d_{x_mu x_mu} + a2/d (Sec. 1, after eq. (2)).
    FD: a dense n_mu x n_mu complex matrix.  Periodic: the diagonal of A_mu in
    Fourier space (Sec. 3.2), returned as a vector."""
    if getattr(p, "mats", None) is not None:
        return np.array(p.mats[mu], dtype=complex)
    n, lo, hi, bc = p.n[mu], p.lo[mu], p.hi[mu], p.bc[mu]
    c = complex(p.a1, p.b1)
    if bc == PERIODIC:
        k = wavenumbers(n, lo, hi)
        return c * (-(k * k)) + p.a2 / p.d
    return c * fd_laplacian(n, lo, hi, bc) + (p.a2 / p.d) * np.eye(n)


def expm(M: np.ndarray) -> np.ndarray:
    """Matrix exponential by Pade scaling and squaring (Al-Mohy & Higham),
    the method the paper uses for the small factors (Sec. 3.1, Sec. 4)."""
    return scipy.linalg.expm(M)


# --------------------------------------------------------------------------
# mu-mode products and the Tucker operator (Sec. 3.1, eqs. kronsumv, Tucker)
# --------------------------------------------------------------------------

def mode_product(U: np.ndarray, M: np.ndarray, mu: int) -> np.ndarray:
    """(U x_mu M)_{i_1..i_mu..i_d} = sum_j M_{i_mu j} U_{i_1..j..i_d}
    (Sec. 3.1, the mu-mode product)."""
    V = np.tensordot(M, U, axes=([1], [mu]))
    return np.moveaxis(V, 0, mu)


def tucker(U: np.ndarray, mats: Sequence[np.ndarray]) -> np.ndarray:
    """U x_1 M_1 x_2 ... x_d M_d (eq. Tucker), applied mode 1 first."""
    for mu, M in enumerate(mats):
        U = mode_product(U, M, mu)
    return U


def kronsumv(U: np.ndarray, mats: Sequence[np.ndarray]) -> np.ndarray:
    """K u = vec(sum_mu U x_mu A_mu)  (eq. kronsumv)."""
    out = np.zeros_like(U, dtype=complex)
    for mu, A in enumerate(mats):
        out = out + mode_product(U, A, mu)
    return out


def kron_sum_dense(mats: Sequence[np.ndarray]) -> np.ndarray:
    """Brute-force K = A_d (+) ... (+) A_1 = sum_mu I x..x A_mu x..x I
    (Sec. 1, eq. (2)) as a dense N x N matrix acting on vec(U)."""
    sizes = [M.shape[0] for M in mats]
    N = int(np.prod(sizes))
    K = np.zeros((N, N), dtype=complex)
    for mu, A in enumerate(mats):
        term = np.ones((1, 1))
        # Kronecker order: A_{(x) mu} = I_d x ... x A_mu x ... x I_1
        for nu in reversed(range(len(mats))):
            term = np.kron(term, A if nu == mu else np.eye(sizes[nu]))
        K += term
    return K


# --------------------------------------------------------------------------
# Linear flows exp(c tau K)
# --------------------------------------------------------------------------

class LinearOperator:
    """Everything the schemes need from K for one problem and step size:
    the action of exp(c tau K) and of K (Sec. 3.1 / 3.2)."""

    def __init__(self, prob, tau: float):
        self.p = as_problem(prob)
        self.tau = float(tau)
        self.A = [direction_matrix(self.p, mu) for mu in range(self.p.d)]
        self._cache = {}

    def factors(self, c: float):
        """exp(c tau A_mu) for every direction, computed once per distinct c
        (Sec. 3.1: the small exponentials are precomputed for constant tau)."""
        key = float(c)
        if key not in self._cache:
            if self.p.periodic:
                self._cache[key] = [np.exp(c * self.tau * a) for a in self.A]
            else:
                self._cache[key] = [expm(c * self.tau * A) for A in self.A]
        return self._cache[key]

    def expK(self, U: np.ndarray, c: float) -> np.ndarray:
        """exp(c tau K) u.  FD: the Tucker operator (eq. Tucker).  Periodic:
        pointwise multiplication by the tensor E in Fourier space (Sec. 3.2),
        with the unnormalised forward FFT and the 1/N inverse."""
        F = self.factors(c)
        if self.p.periodic:
            E = _outer_product(F)
            return np.fft.ifftn(E * np.fft.fftn(U))
        return tucker(U, F)

    def K(self, U: np.ndarray) -> np.ndarray:
        """K u.  FD: eq. kronsumv.  Periodic: pointwise multiplication by the
        symbol tensor (Sec. 3.2) in Fourier space."""
        if self.p.periodic:
            S = _outer_sum(self.A)
            return np.fft.ifftn(S * np.fft.fftn(U))
        return kronsumv(U, self.A)


def _outer_product(vecs):
    out = np.ones(())
    for mu, v in enumerate(vecs):
        shape = [1] * len(vecs)
        shape[mu] = v.shape[0]
        out = out * v.reshape(shape)
    return out


def _outer_sum(vecs):
    out = np.zeros(())
    for mu, v in enumerate(vecs):
        shape = [1] * len(vecs)
        shape[mu] = v.shape[0]
        out = out + v.reshape(shape)
    return out


# --------------------------------------------------------------------------
# Nonlinear part (Sec. 1 eq. (1); Sec. 4.1 eq. exsolcub; Sec. 4.3)
# --------------------------------------------------------------------------

def g(p: OracleProblem, u: np.ndarray) -> np.ndarray:
    """g(u) = (a3 + i b3)|u|^2 u + (a4 + i b4)|u|^4 u (eq. (1))."""
    rho = (u * np.conj(u)).real
    return complex(p.a3, p.b3) * rho * u + complex(p.a4, p.b4) * rho * rho * u


def _lam(x: np.ndarray) -> np.ndarray:
    """Lambda(x) = -log|1 - x| / x, Lambda(0) = 1.  With it the exact flows of
    eq. exsolcub and of the quintic part (Sec. 4.3) read
    u0 * exp((a+ib) r t Lambda(k a r t)), which is the paper's expression for
    a != 0 and stays defined at a = 0 (the paper assumes alpha3 != 0; the
    workloads allow alpha4 = 0 with beta4 != 0).  Series below |x| < 1e-8."""
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-8
    xs = x[small]
    out[small] = 1.0 + xs / 2.0 + xs * xs / 3.0
    xb = x[~small]
    lg = np.empty_like(xb)
    below = xb < 1.0
    lg[below] = np.log1p(-xb[below])
    with np.errstate(divide="ignore"):
        lg[~below] = np.log(xb[~below] - 1.0)
    out[~small] = -lg / xb
    return out


def phi_cubic(p: OracleProblem, u: np.ndarray, t: float) -> np.ndarray:
    """Exact flow of u' = (a3 + i b3)|u|^2 u over time t (eq. exsolcub):
    u(t) = exp(-(a3+i b3)/(2 a3) log|1 - 2 a3 |u0|^2 t|) u0."""
    rho = (u * np.conj(u)).real
    x = 2.0 * p.a3 * rho * t
    return u * np.exp(complex(p.a3, p.b3) * rho * t * _lam(x))


def phi_quintic(p: OracleProblem, u: np.ndarray, t: float) -> np.ndarray:
    """Exact flow of u' = (a4 + i b4)|u|^4 u over time t (Sec. 4.3):
    u(t) = exp(-(a4+i b4)/(4 a4) log|1 - 4 a4 |u0|^4 t|) u0."""
    rho = (u * np.conj(u)).real
    r2 = rho * rho
    x = 4.0 * p.a4 * r2 * t
    return u * np.exp(complex(p.a4, p.b4) * r2 * t * _lam(x))


def rk4_nonlinear(p: OracleProblem, u: np.ndarray, t: float) -> np.ndarray:
    """One classical RK4 step (eq. RK4 with K = 0) of u' = g(u) over time t:
    the approximate nonlinear flow the paper uses for the cubic-quintic model
    (Sec. 4.3 and Sec. 4.4, "a single step of rk4")."""
    k1 = g(p, u)
    k2 = g(p, u + 0.5 * t * k1)
    k3 = g(p, u + 0.5 * t * k2)
    k4 = g(p, u + t * k3)
    return u + (t / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def nonlinear_flow(p: OracleProblem, u: np.ndarray, t: float) -> np.ndarray:
    """phi_t of the splitting schemes (Sec. 2.1): exact for the cubic model
    (eq. exsolcub), one RK4 step for the cubic-quintic model (Sec. 4.3).
    Half-flows of adjacent steps are never merged."""
    if p.cubic:
        return phi_cubic(p, u, t)
    return rk4_nonlinear(p, u, t)


# --------------------------------------------------------------------------
# Time integrators (Sec. 2), written as printed
# --------------------------------------------------------------------------

def step_strang(L: LinearOperator, u):
    """eq. Strang: u_{n+1} = phi_{tau/2}(exp(tau K) phi_{tau/2}(u_n))."""
    p, tau = L.p, L.tau
    return nonlinear_flow(p, L.expK(nonlinear_flow(p, u, tau / 2), 1.0), tau / 2)


def step_split4(L: LinearOperator, u):
    """eq. Richardson (explicit form of eq. richextrap):
    u_{n2}   = phi_{tau/2}(e^{tau K} phi_{tau/2}(u_n))
    u_{n+1}  = 4/3 phi_{tau/4}(e^{tau K/2} phi_{tau/2}(e^{tau K/2} phi_{tau/4}(u_n)))
               - 1/3 u_{n2}
    The middle phi_{tau/2} is one flow of length tau/2."""
    p, tau = L.p, L.tau
    phi = lambda v, t: nonlinear_flow(p, v, t)
    un2 = phi(L.expK(phi(u, tau / 2), 1.0), tau / 2)
    v = phi(L.expK(phi(u, tau / 4), 0.5), tau / 2)
    return (4.0 / 3.0) * phi(L.expK(v, 0.5), tau / 4) - (1.0 / 3.0) * un2


def step_lawson4(L: LinearOperator, u):
    """eq. lawson4, with all six exponential actions as printed (E_1 and
    E_{1/2} applied separately)."""
    p, tau = L.p, L.tau
    gn = g(p, u)
    un2 = L.expK(u + (tau / 2) * gn, 0.5)
    gn2 = g(p, un2)
    un3 = L.expK(u, 0.5) + (tau / 2) * gn2
    gn3 = g(p, un3)
    un4 = L.expK(u, 1.0) + tau * L.expK(gn3, 0.5)
    gn4 = g(p, un4)
    return (L.expK(u + (tau / 6) * gn, 1.0)
            + (tau / 3) * L.expK(gn2 + gn3, 0.5)
            + (tau / 6) * gn4)


def step_lawson2(L: LinearOperator, u):
    """eq. lawson2b (if2)."""
    p, tau = L.p, L.tau
    gn = g(p, u)
    un2 = L.expK(u + tau * gn, 1.0)
    return L.expK(u + (tau / 2) * gn, 1.0) + (tau / 2) * g(p, un2)


def step_rk4(L: LinearOperator, u):
    """eq. RK4 on u' = K u + g(u)."""
    p, tau = L.p, L.tau
    f = lambda v: L.K(v) + g(p, v)
    f1 = f(u)
    f2 = f(u + (tau / 2) * f1)
    f3 = f(u + (tau / 2) * f2)
    f4 = f(u + tau * f3)
    return u + (tau / 6) * (f1 + 2 * f2 + 2 * f3 + f4)


def step_rk2(L: LinearOperator, u):
    """eq. RK2 (Heun) on u' = K u + g(u)."""
    p, tau = L.p, L.tau
    f = lambda v: L.K(v) + g(p, v)
    f1 = f(u)
    f2 = f(u + tau * f1)
    return u + (tau / 2) * (f1 + f2)


def strang3t_step(L: LinearOperator, u, h: float):
    """The three-term Strang step S^3_h of Sec. 4.3 (cubic and quintic parts
    of the nonlinearity split apart, each with its exact flow):
    S^3_h(u) = phi^q_{h/2}(phi^c_{h/2}(e^{hK} phi^c_{h/2}(phi^q_{h/2}(u)))).
    h is tau or tau/2 (the linear flows the operator holds)."""
    p = L.p
    v = phi_cubic(p, phi_quintic(p, u, h / 2), h / 2)
    v = L.expK(v, h / L.tau)
    return phi_quintic(p, phi_cubic(p, v, h / 2), h / 2)


def step_strang3t(L: LinearOperator, u):
    """strang_3t (Sec. 4.3): u_{n+1} = S^3_tau(u_n)."""
    return strang3t_step(L, u, L.tau)


def step_split4_3t(L: LinearOperator, u):
    """split4_3t (Sec. 4.3): the Richardson extrapolation of S^3, as printed
    (the two half steps applied in turn, no flows merged):
    u_{n+1} = 4/3 S^3_{tau/2}(S^3_{tau/2}(u_n)) - 1/3 S^3_tau(u_n)."""
    tau = L.tau
    half = strang3t_step(L, strang3t_step(L, u, tau / 2), tau / 2)
    return (4.0 / 3.0) * half - (1.0 / 3.0) * strang3t_step(L, u, tau)


SCHEMES = {
    "strang": step_strang,
    "split4": step_split4,
    "lawson4": step_lawson4,
    "lawson2": step_lawson2,
    "rk4": step_rk4,
    "rk2": step_rk2,
    "strang3t": step_strang3t,
    "split4_3t": step_split4_3t,
}

ORDERS = {"strang": 2, "split4": 4, "lawson4": 4, "lawson2": 2, "rk4": 4, "rk2": 2, "strang3t": 2, "split4_3t": 4}


def integrate(prob, U0: np.ndarray, tau: float, nsteps: int, scheme: str) -> np.ndarray:
    """Apply ``nsteps`` constant steps of ``scheme`` to U0 (shape n_1..n_d)."""
    L = LinearOperator(prob, tau)
    step = SCHEMES[scheme]
    U = np.array(U0, dtype=complex)
    for _ in range(int(nsteps)):
        U = step(L, U)
    return U


# --------------------------------------------------------------------------
# Error measures (Sec. 4: relative infinity norm; relative 2-norm as well)
# --------------------------------------------------------------------------

def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref)
    return float(np.linalg.norm((np.asarray(x) - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_inf(x: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


def observed_order(steps_a: int, err_a: float, steps_b: int, err_b: float) -> float:
    """Observed order of convergence between two runs to the same final time,
    as the paper's tables report it: log(e_a/e_b) / log(m_b/m_a)."""
    return math.log(err_a / err_b) / math.log(steps_b / steps_a)
