"""Batched instances (cgl_batch_*) against single plans and the FP64 oracle,
and the tile-size autotuner."""
import os

import numpy as np
import pytest
import torch

from oracle import cgl_oracle as O
from paper_2403_02816_gb300 import inputs as I
from paper_2403_02816_gb300 import native as nat

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 2e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2403_02816_gb300 import build as B
    B.build()
    nat.load()
    assert torch.cuda.is_available()


def oprob(p):
    return O.OracleProblem(p.n, p.bc, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)


def mixed_instances(seed=11):
    """Uneven grids (1D, 2D non-square, 3D), Dirichlet/Neumann mixes,
    cubic and cubic-quintic, parameters in the batched workload's ranges."""
    rng = np.random.default_rng(seed)
    shapes = [((48, 57), (0, 1)), ((64,), (1,)), ((33, 20, 9), (1, 0, 1)), ((130, 49), (1, 1)),
              ((50, 50), (0, 0)), ((7, 96), (0, 1)), ((256, 48), (1, 0))]
    probs, fields = [], []
    for k, (n, bc) in enumerate(shapes):
        p = I.random_problem(rng, n, bc, cubic=(k % 2 == 0))
        probs.append(p)
        fields.append(I.u0_bumps(p, rng))
    return probs, fields


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16x3"])
@pytest.mark.parametrize("scheme", ["lawson4", "strang", "split4", "lawson2", "split4_3t"])
def test_batch_equals_single_plans_and_oracle(prec, scheme):
    """BF16x3: the grouped launches run the single plan's kernels per instance
    (same splits, MMA order and epilogue), so batch and single plans agree."""
    probs, fields = mixed_instances()
    tau, nsteps = 0.01, 4
    dt = torch.complex128 if prec == "f64" else torch.complex64
    with nat.Batch(probs, tau, scheme, prec) as b:
        u = b.pack(fields)
        b.step(u, nsteps)
        torch.cuda.synchronize()
        assert b.device_status() == nat.CGL_OK
        got = b.unpack(u)
    for p, U0, G in zip(probs, fields, got):
        with nat.Plan(p, tau, scheme, prec) as plan:
            v = nat.to_device(U0, dt)
            plan.step(v, nsteps)
            single = nat.from_device(v)
        # the same tile code and summation order per point as a single plan
        tol = 1e-13 if prec == "f64" else 1e-6
        assert O.rel_l2(G, single) <= tol
        ref = O.integrate(oprob(p), U0, tau, nsteps, scheme)
        assert O.rel_l2(G, ref) <= TOL[prec], (p.n, O.rel_l2(G, ref))


@pytest.mark.parametrize("prec", ["f32", "bf16x3"])
def test_batch_graph_follows_new_field_pointer(prec):
    probs, fields = mixed_instances(3)
    with nat.Batch(probs[:3], 0.01, "lawson4", prec) as b:
        a = b.pack(fields[:3])
        c = b.pack(fields[:3])
        b.step(a, 2)
        b.step(c, 2)
        torch.cuda.synchronize()
        assert torch.equal(a, c)


@pytest.mark.parametrize("prec", ["f32", "bf16x3"])
def test_batched_workload_subset_against_oracle_full_run(prec):
    """The 512-instance workload's first 4 instances (complex64, Lawson4,
    tau = 0.01, 200 steps) inside a 16-instance batch, against the oracle."""
    probs = I.batched_problems(16)
    fields = [I.u0_bumps(p, np.random.Generator(np.random.PCG64(I.SEED_BASE + 3 + 1000 * i)))
              for i, p in enumerate(probs)]
    with nat.Batch(probs, 0.01, "lawson4", prec) as b:
        u = b.pack(fields)
        b.step(u, 200)
        torch.cuda.synchronize()
        assert b.device_status() == nat.CGL_OK
        got = b.unpack(u)
    for i in range(4):
        ref = O.integrate(oprob(probs[i]), fields[i], 0.01, 200, "lawson4")
        assert O.rel_l2(got[i], ref) <= 1e-4, (i, probs[i].n, O.rel_l2(got[i], ref))


def test_autotuner_returns_admissible_tiles_and_caches(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CGL_AUTOTUNE_CACHE", str(cache))
    seen = []
    for n, contiguous in [(37, 1), (211, 0)]:
        tb, ms = nat.cgl_autotune_mode_tile(n, contiguous, nat.CGL_F32, 2)
        assert tb in (2, 4, 8, 16, 32, 64) and ms > 0
        seen.append((n, tb))
        # a second call is served from the in-process cache
        assert nat.cgl_autotune_mode_tile(n, contiguous, nat.CGL_F32, 2)[0] == tb
    tb, _ = nat.cgl_autotune_mode_tile(1021, 1, nat.CGL_F64, 1)
    assert tb in (2, 4)  # 96 KiB of shared memory holds at most 5 fibers of 1021 complex128
    assert any(l.startswith("1021 1 0 1 ") for l in cache.read_text().splitlines())
