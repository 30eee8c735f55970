"""GPU parity for the mixed-radix FFT passes (periodic sizes 2^a 3^b 5^c 7^d)
and the coupled two-field system (Sec. 4.5, eq. coupled) against the FP64
oracles."""
import numpy as np
import pytest
import torch

from oracle import cgl_oracle as O
from oracle import coupled_oracle as C
from paper_2403_02816_gb300 import inputs as I
from paper_2403_02816_gb300 import native as nat

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 2e-5}
DT = {"f64": torch.complex128, "f32": torch.complex64}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2403_02816_gb300 import build as B
    B.build()
    nat.load()
    assert torch.cuda.is_available()


def oprob(p):
    return O.OracleProblem(p.n, p.bc, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)


def cprob(p):
    return C.CoupledProblem(p.n, p.lo, p.hi, p.a0, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4, p.a5)


def check(got, ref, prec, what=""):
    err, einf = O.rel_l2(got, ref), O.rel_inf(got, ref)
    # per-value bounds: they hold in relative L2 and relative inf alike
    assert err <= TOL[prec] and einf <= TOL[prec], (what, err, einf)


# ------------------------------------------------------------ mixed radix, one field

MR_SHAPES = [(12,), (45,), (700,), (60, 14), (21, 10), (70, 35), (9, 25, 14), (1400, 4)]


@pytest.mark.parametrize("n", MR_SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mixed_radix_linear_flow(n, prec):
    """exp(c tau K) on periodic sizes with factors 3, 5, 7 (odd sizes included:
    signed frequencies up to (n-1)/2) against the oracle's FFT form."""
    rng = np.random.default_rng(3)
    d = len(n)
    p = I.Problem(tuple(n), (I.PERIODIC,) * d, (0.0,) * d, tuple(10.0 + 3 * m for m in range(d)),
                  0.3, 0.7, -0.2, 1.0, 0.5, -0.1, 0.2)
    U = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    L = O.LinearOperator(oprob(p), 0.013)
    with nat.Plan(p, 0.013, "split4", prec) as plan:
        for c in (1.0, 0.5):
            u = nat.to_device(U, DT[prec])
            plan.linear_flow(u, c)
            check(nat.from_device(u), L.expK(U, c), prec, "c=%g" % c)


@pytest.mark.parametrize("n", [(60, 14), (45,), (21, 10, 6)])
@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "rk4"])
def test_mixed_radix_schemes(n, scheme):
    rng = np.random.default_rng(4)
    d = len(n)
    p = I.Problem(tuple(n), (I.PERIODIC,) * d, (0.0,) * d, tuple(8.0 + 2 * m for m in range(d)),
                  0.3, 0.7, -0.2, 1.0, 0.5, -0.1, 0.2)
    U0 = 0.5 * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n))
    tau = 0.002 if scheme == "rk4" else 0.01
    ref = O.integrate(oprob(p), U0, tau, 4, scheme)
    with nat.Plan(p, tau, scheme, "f64") as plan:
        u = nat.to_device(U0, torch.complex128)
        plan.step(u, 4)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        check(nat.from_device(u), ref, "f64", scheme)


# ------------------------------------------------------------ coupled system

COUPLED_SHAPES = [(32, 16), (70, 35), (56, 20), (30, 12, 7)]


def small_coupled(n):
    d = len(n)
    base = I.coupled_problem()
    return I.CoupledProblem(tuple(n), (0.0,) * d, tuple([7.0, 3.5, 2.0][:d]), base.a0, base.a1, base.b1, base.a2,
                            base.a3, base.b3, base.a4, base.b4, base.a5)


def coupled_data(p, rng):
    X = np.meshgrid(*[np.arange(m) / m for m in p.n], indexing="ij")
    u = 0.8 * np.exp(2j * np.pi * X[0]) + 0.3 * np.cos(2 * np.pi * X[1])
    v = 0.6 * np.exp(-2j * np.pi * X[1]) + 0.2j * np.sin(4 * np.pi * X[0])
    W = np.stack([u, v]) * (1 + 0.05 * (rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)))
    return W


@pytest.mark.parametrize("n", COUPLED_SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coupled_linear_flow(n, prec):
    """Block-diagonal exp(c tau K): each field with its own advection sign."""
    rng = np.random.default_rng(5)
    p = small_coupled(n)
    W = coupled_data(p, rng)
    L = C.CoupledLinear(cprob(p), 0.02)
    with nat.CoupledPlan(p, 0.02, "split4", prec) as plan:
        for c in (1.0, 0.5):
            w = nat.to_device_pair(W, DT[prec])
            plan.linear_flow(w, c)
            check(nat.from_device_pair(w), L.expK(W, c), prec, "c=%g" % c)


@pytest.mark.parametrize("n", COUPLED_SHAPES)
@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2", "rk4", "rk2"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coupled_schemes_match_oracle(n, scheme, prec):
    rng = np.random.default_rng(6)
    p = small_coupled(n)
    W0 = coupled_data(p, rng)
    # explicit Runge-Kutta: a step inside its stability limit on these grids
    tau, nsteps = (0.001, 5) if scheme.startswith("rk") else (0.01, 5)
    ref = C.integrate(cprob(p), W0, tau, nsteps, scheme)
    with nat.CoupledPlan(p, tau, scheme, prec) as plan:
        w = nat.to_device_pair(W0, DT[prec])
        plan.step(w, nsteps)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        check(nat.from_device_pair(w), ref, prec, scheme)


def test_coupled_mirror_symmetry_on_gpu():
    """v0 = u0 mirrored in x1 keeps v = mirrored u (the Nyquist advection
    symbol is 0), in the GPU result as in the oracle."""
    rng = np.random.default_rng(7)
    p = small_coupled((40, 12))
    u0 = coupled_data(p, rng)[0]
    mirror = lambda a: np.roll(a[::-1, :], 1, axis=0)
    W0 = np.stack([u0, mirror(u0)])
    with nat.CoupledPlan(p, 0.01, "split4", "f64") as plan:
        w = nat.to_device_pair(W0, torch.complex128)
        plan.step(w, 6)
        got = nat.from_device_pair(w)
    assert np.max(np.abs(got[1] - mirror(got[0]))) < 1e-12 * np.max(np.abs(got))


@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2", "rk4", "rk2"])
def test_coupled_paper_grid_700x350(scheme):
    """The paper's 700 x 350 grid, parameters and soliton-pair data, 3 steps
    of tau = 3/500 (its coarsest split4 step; 3/2562, its finest RK step, for
    the explicit schemes), FP64 against the oracle."""
    p = I.coupled_problem()
    W0 = I.coupled_u0(p)
    tau, nsteps = (3.0 / 2562 if scheme.startswith("rk") else 3.0 / 500), 3
    ref = C.integrate(cprob(p), W0, tau, nsteps, scheme)
    with nat.CoupledPlan(p, tau, scheme, "f64") as plan:
        w = nat.to_device_pair(W0, torch.complex128)
        plan.step(w, nsteps)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        check(nat.from_device_pair(w), ref, "f64", scheme)


# ------------------------------------------------------------ edge sizes

@pytest.mark.parametrize("n", [(2025,), (1715, 2), (1536, 3), (1000,)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_mixed_radix_largest_sizes(n, prec):
    """Mixed-radix passes at the size limit: 2025 = 3^4 5^2 (odd), 1715 = 5 7^3,
    1536 = 2^9 3, 1000 = 2^3 5^3 (one pencil per CTA, the largest twiddle
    tables)."""
    rng = np.random.default_rng(9)
    d = len(n)
    p = I.Problem(tuple(n), (I.PERIODIC,) * d, (0.0,) * d, tuple(30.0 + 5 * m for m in range(d)),
                  0.3, 0.7, -0.2, 1.0, 0.5, -0.1, 0.2)
    U = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    L = O.LinearOperator(oprob(p), 0.013)
    with nat.Plan(p, 0.013, "split4", prec) as plan:
        u = nat.to_device(U, DT[prec])
        plan.linear_flow(u, 0.5)
        check(nat.from_device(u), L.expK(U, 0.5), prec, "n=%s" % (n,))
        U0 = 0.5 * U
        ref = O.integrate(oprob(p), U0, 0.013, 2, "split4")  # the plan's step
        u = nat.to_device(U0, DT[prec])
        plan.step(u, 2)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        check(nat.from_device(u), ref, prec, "split4 n=%s" % (n,))


@pytest.mark.parametrize("n", [(140,), (20, 15, 14)])
@pytest.mark.parametrize("scheme", ["lawson4", "rk4", "split4"])
def test_coupled_1d_and_3d(n, scheme):
    """The coupled system in one and three dimensions (the advection acts on
    direction 1 only)."""
    rng = np.random.default_rng(10)
    d = len(n)
    base = I.coupled_problem()
    p = I.CoupledProblem(tuple(n), (0.0,) * d, tuple([14.0, 3.0, 2.8][:d]), base.a0, base.a1, base.b1, base.a2,
                         base.a3, base.b3, base.a4, base.b4, base.a5)
    shape = tuple(n)
    W0 = 0.6 * (1 + 0.1 * (rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)))
    tau = 0.001 if scheme == "rk4" else 0.01
    ref = C.integrate(cprob(p), W0, tau, 4, scheme)
    with nat.CoupledPlan(p, tau, scheme, "f64") as plan:
        w = nat.to_device_pair(W0, torch.complex128)
        plan.step(w, 4)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        check(nat.from_device_pair(w), ref, "f64", scheme)
