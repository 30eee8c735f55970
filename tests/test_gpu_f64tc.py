"""CGL_F64_TC: the FP64-accurate mu-mode products on the tensor cores (Ozaki
splitting into exact BF16 digits) against the FP64 oracle, through the C ABI.

Tolerances are the FP64 path's: relative L2 <= 1e-11 for runs; a single
linear flow exp(c tau K) is held to 1e-12 (each digit product is exact and
the truncated digit products are below 2^-46 of the operands' row scales, so
one Tucker operator lands near 1e-14).
"""
import numpy as np
import pytest
import torch

from oracle import cgl_oracle as O
from paper_2403_02816_gb300 import inputs as I
from paper_2403_02816_gb300 import native as nat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2403_02816_gb300 import build as B
    B.build()
    nat.load()
    assert torch.cuda.is_available()


def oprob(p):
    return O.OracleProblem(p.n, p.bc, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)


def run_gpu(p, U0, tau, nsteps, scheme, prec="f64tc"):
    with nat.Plan(p, tau, scheme, prec) as plan:
        u = nat.to_device(U0, torch.complex128)
        plan.step(u, nsteps)
        torch.cuda.synchronize()
        assert plan.device_status() == nat.CGL_OK
        return nat.from_device(u)


def rand_problem(seed, n, bc, cubic=True):
    rng = np.random.default_rng(seed)
    return I.random_problem(rng, n, bc, cubic=cubic), rng


def smooth_data(p, rng, amp=0.5):
    X = I.mesh(p)
    r2 = sum(x * x for x in X)
    L2 = max((h - l) for l, h in zip(p.lo, p.hi)) ** 2
    return amp * (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)) * np.exp(-8 * r2 / L2)


# every mode position with a ragged tile (Q or P not a multiple of 128), n
# not a multiple of 16, np <= 64 (one row block) and np > 64 (several
# blocks of 64 rows, the last one partly past np), the 256 maximum
SHAPES = [((16,), (0,)), ((64, 64), (0, 0)), ((37,), (1,)), ((256,), (0,)), ((50, 77), (0, 1)),
          ((128, 16, 80), (0, 1, 1)), ((130, 100), (1, 0)), ((20, 6, 230), (0, 1, 1)), ((3, 256), (1, 1)),
          ((256, 2, 7), (0, 1, 0)), ((2,), (0,)), ((64, 150), (1, 1))]


@pytest.mark.parametrize("n,bc", SHAPES)
def test_linear_flow(n, bc):
    p, rng = rand_problem(5, n, bc)
    tau = 0.013
    U = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    L = O.LinearOperator(oprob(p), tau)
    with nat.Plan(p, tau, "split4", "f64tc") as plan:
        for c in (1.0, 0.5):
            u = nat.to_device(U, torch.complex128)
            plan.linear_flow(u, c)
            torch.cuda.synchronize()
            assert plan.device_status() == nat.CGL_OK
            got = nat.from_device(u)
            e = O.rel_l2(got, L.expK(U, c))
            assert e <= 1e-12, (n, c, e, O.rel_inf(got, L.expK(U, c)))


def test_product_equals_fp64_product_of_the_plan_factors():
    """The Tucker operator on the tensor cores against the same product in
    FP64 (numpy) with the plan's own FP64 factors, isolating the digit
    arithmetic from the factor computation.  Each of the K = 2n products of
    a sum is truncated below 2^-46 of the product of its row scales (the
    per-fiber and per-row powers of two above the largest entries), so a
    sum of random-sign terms errs by about sqrt(K) 2^-46 of the scales, a
    few 1e-13 relative to the result; bound 1e-12 (as one linear flow)."""
    for n, bc in (((48, 7), (0, 1)), ((256, 40), (1, 0)), ((30, 20, 70), (1, 1, 0))):
        p, rng = rand_problem(3, n, bc)
        U = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
        with nat.Plan(p, 0.01, "strang", "f64tc") as plan:
            fac = [plan.factor(1.0, mu) for mu in range(p.d)]
            u = nat.to_device(U, torch.complex128)
            plan.linear_flow(u, 1.0)
            got = nat.from_device(u)
        want = U
        for mu, F in enumerate(fac):
            want = np.moveaxis(np.tensordot(F, want, axes=([1], [mu])), 0, mu)
        assert O.rel_l2(got, want) <= 1e-12, (n, O.rel_l2(got, want))


SCHEME_CASES = [((128, 32), (0, 1)), ((128, 16, 32), (1, 0, 1)), ((64,), (0,)), ((50, 33), (0, 1)),
                ((20, 12, 9), (1, 0, 1))]


@pytest.mark.parametrize("n,bc", SCHEME_CASES)
@pytest.mark.parametrize("cubic", [True, False])
def test_schemes_match_oracle(n, bc, cubic):
    p, rng = rand_problem(6, n, bc, cubic=cubic)
    U0 = smooth_data(p, rng, amp=0.8)
    tau, nsteps = 0.004, 5
    for s in ("strang", "split4", "lawson4", "lawson2", "strang3t", "split4_3t", "rk4", "rk2"):
        ref = O.integrate(oprob(p), U0, tau, nsteps, s)
        got = run_gpu(p, U0, tau, nsteps, s)
        e, einf = O.rel_l2(got, ref), O.rel_inf(got, ref)
        assert e <= 1e-11 and einf <= 1e-11, (s, cubic, e, einf)


def test_workload_2d_dirichlet_full_run():
    """The 64x64 Dirichlet FP64 parity workload (tau = 0.01, 200 steps of
    Strang and of Lawson4) with the mode products on the tensor cores."""
    w = I.workload_2d_dirichlet()
    U0 = I.u0_2d_dirichlet(w)
    for s in w.schemes:
        ref = O.integrate(oprob(w.prob), U0, w.tau, w.nsteps, s)
        got = run_gpu(w.prob, U0, w.tau, w.nsteps, s)
        e2, einf = O.rel_l2(got, ref), O.rel_inf(got, ref)
        assert e2 <= 1e-11 and einf <= 1e-11, (s, e2, einf)


def test_workload_3d_neumann_full_size():
    """3D cubic Neumann 256^3, Lawson4, tau = 0.01, 2 steps against the
    oracle at full size (the launch configuration the benchmark times)."""
    w = I.workload_3d_neumann()
    U0 = I.u0_3d_neumann(w)
    ref = O.integrate(oprob(w.prob), U0, w.tau, 2, "lawson4")
    got = run_gpu(w.prob, U0, w.tau, 2, "lawson4")
    e2, einf = O.rel_l2(got, ref), O.rel_inf(got, ref)
    assert e2 <= 1e-11 and einf <= 1e-11, (e2, einf)


def test_deterministic_and_equal_to_fp64_path_within_bound():
    """Integer digit products make the pass independent of accumulation
    order: two runs give identical bytes; and the result agrees with the
    FP64 SIMT path."""
    p, rng = rand_problem(8, (128, 64, 48), (1, 0, 1), cubic=True)
    U0 = smooth_data(p, rng, amp=0.8)
    runs = [run_gpu(p, U0, 0.004, 4, "lawson4") for _ in range(2)]
    assert runs[0].tobytes() == runs[1].tobytes()
    simt = run_gpu(p, U0, 0.004, 4, "lawson4", "f64")
    assert O.rel_l2(runs[0], simt) <= 1e-12


@pytest.mark.parametrize("n,bc", [((128, 300), (0, 0)), ((8, 8), (2, 2))])
def test_rejects_unsupported_shapes(n, bc):
    p, _ = rand_problem(5, n, bc)
    with pytest.raises(nat.CglError) as ei:
        nat.Plan(p, 0.01, "strang", "f64tc")
    assert ei.value.status == nat.CGL_EUNSUPPORTED


def test_batches_do_not_take_it():
    p, _ = rand_problem(5, (16, 16), (0, 0))
    with pytest.raises(nat.CglError) as ei:
        nat.Batch([p], 0.01, "lawson4", "f64tc")
    assert ei.value.status == nat.CGL_EUNSUPPORTED
