"""Seeded synthetic workloads for the CGL integrators.

This module holds problem descriptions and initial data only: no step of the
method's arithmetic lives here.  It is the one module that both the CUDA
path's callers (tests, bench) and the CPU oracle's callers use, so that both
sides see bit-identical inputs.

Arrays are complex128 of shape (n_1, ..., n_d) indexed like the paper's
U_{i_1..i_d}; ``device_layout`` turns one into the flat n_1-fastest order the
C ABI takes (the paper's vec(U), Sec. 3.1).

Seeds: numpy PCG64, seed = 2403028160 + workload index (0..4), so every run
regenerates the same fields.  "N(0,1) complex noise" means independent
standard normal real and imaginary parts, drawn as two arrays of N values in
vec order (real first).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Tuple

import numpy as np

SEED_BASE = 2403028160

DIRICHLET, NEUMANN, PERIODIC = 0, 1, 2
BC_NAMES = {DIRICHLET: "D", NEUMANN: "N", PERIODIC: "P"}


@dataclass
class Problem:
    """Parameters of eq. (1) on a box with per-direction boundary conditions."""

    n: Tuple[int, ...]
    bc: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    a1: float
    b1: float
    a2: float
    a3: float
    b3: float
    a4: float = 0.0
    b4: float = 0.0

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def periodic(self) -> bool:
        return all(b == PERIODIC for b in self.bc)

    def with_n(self, n) -> "Problem":
        return replace(self, n=tuple(int(v) for v in n))


def nodes(n: int, lo: float, hi: float, bc: int) -> np.ndarray:
    """Grid node coordinates of one direction.
    DIRICHLET: interior nodes lo + j h, j = 1..n, h = (hi-lo)/(n+1).
    NEUMANN:   lo + j h, j = 0..n-1, h = (hi-lo)/(n-1) (both ends included).
    PERIODIC:  lo + j h, j = 0..n-1, h = (hi-lo)/n."""
    if bc == DIRICHLET:
        h = (hi - lo) / (n + 1)
        return lo + h * np.arange(1, n + 1)
    if bc == NEUMANN:
        h = (hi - lo) / (n - 1)
        return lo + h * np.arange(n)
    h = (hi - lo) / n
    return lo + h * np.arange(n)


def mesh(prob: Problem):
    """Coordinate arrays X_mu of shape (n_1, ..., n_d)."""
    axes = [nodes(prob.n[m], prob.lo[m], prob.hi[m], prob.bc[m]) for m in range(prob.d)]
    return np.meshgrid(*axes, indexing="ij")


def complex_noise(rng: np.random.Generator, n) -> np.ndarray:
    """Independent N(0,1) real and imaginary parts, drawn in vec order."""
    N = int(np.prod(n))
    re = rng.standard_normal(N)
    im = rng.standard_normal(N)
    return (re + 1j * im).reshape(tuple(n), order="F")


def device_layout(U: np.ndarray) -> np.ndarray:
    """Flat vec(U) (n_1 fastest), contiguous complex128."""
    return np.ascontiguousarray(U.reshape(-1, order="F"))


def from_device_layout(u: np.ndarray, n) -> np.ndarray:
    return np.asarray(u).reshape(tuple(n), order="F")


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    prob: Problem
    tau: float
    nsteps: int
    schemes: Tuple[str, ...]
    precision: str
    seed: int
    extra: dict = field(default_factory=dict)


def workload_2d_dirichlet(n: int = 64) -> Workload:
    """2D cubic CGL, homogeneous Dirichlet, (-10,10)^2, 2nd-order FD,
    64 x 64 interior grid, complex128; tau = 0.01, 200 steps."""
    prob = Problem((n, n), (DIRICHLET, DIRICHLET), (-10.0, -10.0), (10.0, 10.0),
                   a1=1.0, b1=0.5, a2=1.0, a3=-1.0, b3=1.2)
    return Workload("2d_cubic_dirichlet_fd2_64x64_c128", prob, 0.01, 200,
                    ("strang", "lawson4"), "f64", SEED_BASE + 0)


def u0_2d_dirichlet(w: Workload) -> np.ndarray:
    """0.1 * (complex N(0,1) field) * exp(-(x^2 + y^2)/8)."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    X = mesh(w.prob)
    r2 = sum(x * x for x in X)
    return 0.1 * complex_noise(rng, w.prob.n) * np.exp(-r2 / 8.0)


def workload_3d_periodic(n: int = 128) -> Workload:
    """3D cubic-quintic CGL, periodic, (-20,20)^3, Fourier 128^3, complex128;
    tau = 0.005, 500 steps; split4 vs Strang vs RK4."""
    prob = Problem((n, n, n), (PERIODIC,) * 3, (-20.0,) * 3, (20.0,) * 3,
                   a1=0.5, b1=0.5, a2=-0.1, a3=1.0, b3=1.0, a4=-0.1, b4=-0.1)
    return Workload("3d_cubicquintic_periodic_fourier_128^3_c128", prob, 0.005, 500,
                    ("split4", "strang", "rk4"), "f64", SEED_BASE + 1)


def u0_3d_periodic(w: Workload) -> np.ndarray:
    """1.2 * sech(r/2) + 1e-3 * (complex N(0,1) field), r = |x|."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    X = mesh(w.prob)
    r = np.sqrt(sum(x * x for x in X))
    return 1.2 / np.cosh(r / 2.0) + 1e-3 * complex_noise(rng, w.prob.n)


def workload_3d_neumann(n: int = 256) -> Workload:
    """3D cubic CGL, homogeneous Neumann, (-10,10)^3, 2nd-order FD 256^3;
    parameters as the 2D Dirichlet workload; tau = 0.01, 100 steps (T = 1);
    Lawson4 in complex64 (FP32 and BF16x3 GEMMs) against FP64."""
    prob = Problem((n, n, n), (NEUMANN,) * 3, (-10.0,) * 3, (10.0,) * 3,
                   a1=1.0, b1=0.5, a2=1.0, a3=-1.0, b3=1.2)
    return Workload("3d_cubic_neumann_fd2_256^3", prob, 0.01, 100,
                    ("lawson4", "strang"), "f32", SEED_BASE + 2)


def u0_3d_neumann(w: Workload, ell: float = 2.0, rms: float = 0.1) -> np.ndarray:
    """Smooth random field: complex white noise filtered in Fourier space by
    exp(-|kappa|^2 ell^2 / 4) (a Gaussian covariance of correlation length
    ell), rescaled to RMS ``rms``.  The filter treats the node grid as
    periodic with spacing h."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    p = w.prob
    xi = complex_noise(rng, p.n)
    spec = np.fft.fftn(xi)
    filt = np.ones(())
    for m in range(p.d):
        h = (p.hi[m] - p.lo[m]) / (p.n[m] - 1)
        k = 2.0 * np.pi * np.fft.fftfreq(p.n[m], d=h)
        shape = [1] * p.d
        shape[m] = p.n[m]
        filt = filt * np.exp(-(k * k) * ell * ell / 4.0).reshape(shape)
    U = np.fft.ifftn(spec * filt)
    return U * (rms / np.sqrt(np.mean(np.abs(U) ** 2)))


def batched_problems(count: int = 512, seed: int = SEED_BASE + 3):
    """Independent 2D cubic / cubic-quintic instances: grids uniform in
    48..256 per direction, per-direction Dirichlet/Neumann, a1 in [0.2,2],
    b1 in [-2,2], a2 in [0.1,1], a3 in [-2,-0.5], b3 in [-2,2],
    a4 in {0,-0.1}, b4 in {0,0.1}, domain (-10,10)^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.integers(48, 257, size=2))
        bc = tuple(int(v) for v in rng.integers(0, 2, size=2))
        probs.append(Problem(n, bc, (-10.0, -10.0), (10.0, 10.0),
                             a1=float(rng.uniform(0.2, 2.0)),
                             b1=float(rng.uniform(-2.0, 2.0)),
                             a2=float(rng.uniform(0.1, 1.0)),
                             a3=float(rng.uniform(-2.0, -0.5)),
                             b3=float(rng.uniform(-2.0, 2.0)),
                             a4=float(rng.choice([0.0, -0.1])),
                             b4=float(rng.choice([0.0, 0.1]))))
    return probs


def u0_bumps(prob: Problem, rng: np.random.Generator, count: int = 3) -> np.ndarray:
    """Sum of ``count`` Gaussian bumps A exp(-|x-c|^2/(2 s^2)) e^{i theta},
    A ~ U[0.2,1], s ~ U[1,3], c uniform in the central 60% of the box,
    theta ~ U[0, 2 pi)."""
    X = mesh(prob)
    U = np.zeros(prob.n, dtype=complex)
    for _ in range(count):
        A = rng.uniform(0.2, 1.0)
        s = rng.uniform(1.0, 3.0)
        c = [prob.lo[m] + (prob.hi[m] - prob.lo[m]) * rng.uniform(0.2, 0.8)
             for m in range(prob.d)]
        th = rng.uniform(0.0, 2.0 * np.pi)
        r2 = sum((X[m] - c[m]) ** 2 for m in range(prob.d))
        U = U + A * np.exp(-r2 / (2 * s * s)) * np.exp(1j * th)
    return U


def random_problem(rng: np.random.Generator, n, bc, cubic: bool = True,
                   lo: float = -10.0, hi: float = 10.0) -> Problem:
    """A small random test problem (parameter ranges of the batched workload)."""
    d = len(n)
    return Problem(tuple(n), tuple(bc), (lo,) * d, (hi,) * d,
                   a1=float(rng.uniform(0.2, 2.0)), b1=float(rng.uniform(-2.0, 2.0)),
                   a2=float(rng.uniform(0.1, 1.0)), a3=float(rng.uniform(-2.0, -0.5)),
                   b3=float(rng.uniform(-2.0, 2.0)),
                   a4=0.0 if cubic else -0.1, b4=0.0 if cubic else 0.1)


def plane_wave_data(prob: Problem, m_vec, amp: float) -> np.ndarray:
    """amp * exp(i k.x) with k_mu = 2 pi m_mu / (hi_mu - lo_mu) on the
    periodic grid (initial data only; its evolution is not computed here)."""
    X = mesh(prob)
    phase = sum(2 * np.pi * m_vec[mu] / (prob.hi[mu] - prob.lo[mu]) * X[mu]
                for mu in range(prob.d))
    return amp * np.exp(1j * phase)


# --------------------------------------------------------------------------
# Coupled two-field system (Sec. 4.5, eq. coupled)
# --------------------------------------------------------------------------

@dataclass
class CoupledProblem:
    """Parameters of eq. (coupled), periodic in every direction."""

    n: Tuple[int, ...]
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    a0: float
    a1: float
    b1: float
    a2: float
    a3: float
    b3: float
    a4: float
    b4: float
    a5: float

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def bc(self):
        return (PERIODIC,) * self.d

    @property
    def periodic(self) -> bool:
        return True


def coupled_problem(n1: int = 700, n2: int = 350) -> CoupledProblem:
    """The paper's coupled workload (Sec. 4.5): (0, 70) x (0, 35), a0 = -0.4,
    a5 = 0.5, a1 = 0.125, b1 = 0.5, a2 = -0.9, a3 = 1, b3 = 0.8, a4 = -0.1,
    b4 = -0.6, n = 700 x 350 (other sizes keep the domain)."""
    return CoupledProblem((n1, n2), (0.0, 0.0), (70.0, 35.0), -0.4, 0.125, 0.5, -0.9, 1.0, 0.8, -0.1, -0.6, 0.5)


def coupled_u0(prob: CoupledProblem, seed: int = SEED_BASE + 5) -> np.ndarray:
    """Two quasi-1D solitons approaching each other: u0(x1, x2) = w0(x1) and
    v0(x1, x2) = w0(L1 - x1), w0 = delta exp(-(x1 - chi)^2 / (2 sigma^2)) with
    the paper's delta = 2.25, chi = 17.5, sigma = 2.5 (the seed of its 1D
    relaxation run, standing in for the relaxed soliton), times (1 + 1e-3 xi)
    with xi complex N(0,1) noise so the x2 direction is not exactly uniform.
    Returns W of shape (2, n1, n2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x1 = nodes(prob.n[0], prob.lo[0], prob.hi[0], PERIODIC)
    L1 = prob.hi[0] - prob.lo[0]
    w = lambda x: 2.25 * np.exp(-((x - 17.5) ** 2) / (2 * 2.5 ** 2))
    shape = tuple(prob.n)
    u = w(x1)[:, None] * np.ones(shape[1:])[None, :]
    v = w(L1 - x1)[:, None] * np.ones(shape[1:])[None, :]
    u = u * (1 + 1e-3 * complex_noise(rng, shape))
    v = v * (1 + 1e-3 * complex_noise(rng, shape))
    return np.stack([u, v]).astype(complex)
