"""Learned corrector of a coarse exponential step, trained on trajectories of
the fine method (2D periodic cubic CGL, 128 x 128, (-10,10)^2).

  fine   : Lawson4 (eq. lawson4), complex128, tau_f = 0.002   (training target and judge)
  coarse : Lawson4, complex64,  tau_c = 0.016 = 8 tau_f
  corrected coarse step: u_{n+1} = C(u_n) + N(x_n)  (cgl_corrector_*)

Parameters per trajectory are drawn from the batched workload's ranges with
a4 = b4 = 0 (cubic): a1 in [0.2,2], b1 in [-2,2], a2 in [0.1,1], a3 in
[-2,-0.5], b3 in [-2,2]; initial data are three random Gaussian bumps.  A
trajectory contributes `snaps` training pairs (u_n, C(u_n), F^8(u_n)) at fine
steps 0, 312, 624, ...  Evaluation runs held-out trajectories to
t = 312 tau_c = 4.992 with and without the correction and compares both with
the fine result.

Every numerical step runs in the library's kernels (plans and corrector);
torch holds device memory and converts between complex128 and complex64
storage.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import native as nat

N = 128
FINE_TAU = 0.002
COARSE_TAU = 0.016
SUB = 8                 # fine steps per coarse step
COARSE_STEPS = 312      # t = 4.992
SEED = I.SEED_BASE + 4


def problem(par, n=N):
    a1, b1, a2, a3, b3 = par
    return I.Problem((n, n), (I.PERIODIC, I.PERIODIC), (-10.0, -10.0), (10.0, 10.0),
                     a1=a1, b1=b1, a2=a2, a3=a3, b3=b3)


def sample(rng, n=N):
    par = (float(rng.uniform(0.2, 2.0)), float(rng.uniform(-2.0, 2.0)), float(rng.uniform(0.1, 1.0)),
           float(rng.uniform(-2.0, -0.5)), float(rng.uniform(-2.0, 2.0)))
    p = problem(par, n)
    return par, p, I.u0_bumps(p, rng)


class Dataset:
    """Device tensors: un, coarse, target (complex64 [P, n, n]), params (float32 [P, 5])."""

    def __init__(self, ntraj, snaps=8, seed=SEED, n=N, device="cuda", concurrency=32, sub=SUB,
                 coarse_steps=COARSE_STEPS):
        """Trajectories run `concurrency` at a time, each on its own CUDA stream
        (one 128^2 instance fills only a few SMs).  The coarse step is `sub`
        fine steps long; snapshots are spread over `coarse_steps` coarse steps.
        Besides the complex64 coarse step, `coarse64_rms` records the RMS of
        the complex128 coarse step's difference to the fine result (the part
        of the correction that does not come from FP32 rounding)."""
        import torch
        P = ntraj * snaps
        self.n = n
        self.un = torch.empty((P, n, n), dtype=torch.complex64, device=device)
        self.coarse = torch.empty_like(self.un)
        self.target = torch.empty_like(self.un)
        host_params = np.empty((P, 5), dtype=np.float32)
        stride = coarse_steps * sub // snaps
        self.sub = sub
        tru_parts = []  # device scalars, summed after the last synchronisation
        streams = [torch.cuda.Stream() for _ in range(min(concurrency, ntraj))]
        t0 = time.perf_counter()
        for g0 in range(0, ntraj, len(streams)):
            group = []
            for gi, i in enumerate(range(g0, min(ntraj, g0 + len(streams)))):
                s = streams[gi]
                rng = np.random.Generator(np.random.PCG64(seed + 1000 * i))
                par, p, U0 = sample(rng, n)
                fine = nat.Plan(p, FINE_TAU, "lawson4", "f64", stream=s)
                crs = nat.Plan(p, FINE_TAU * sub, "lawson4", "f32", stream=s)
                crs64 = nat.Plan(p, FINE_TAU * sub, "lawson4", "f64", stream=s)
                with torch.cuda.stream(s):
                    u = nat.to_device(U0, torch.complex128, device)
                    v = torch.empty_like(u)
                    c = torch.empty((n, n), dtype=torch.complex64, device=device)
                    w = torch.empty_like(u)
                group.append((s, fine, crs, crs64, u, v, c, w, i))
                host_params[i * snaps:(i + 1) * snaps] = par
            for sn in range(snaps):
                for s, fine, crs, crs64, u, v, c, w, i in group:
                    k = i * snaps + sn
                    with torch.cuda.stream(s):
                        if sn > 0:
                            fine.step(u, stride, stream=s)
                        self.un[k].copy_(u)
                        v.copy_(u)
                        fine.step(v, sub, stream=s)
                        self.target[k].copy_(v)
                        c.copy_(self.un[k])
                        crs.step(c, 1, stream=s)
                        self.coarse[k].copy_(c)
                        w.copy_(u)
                        crs64.step(w, 1, stream=s)
                        w.sub_(v)
                        tru_parts.append(w.abs().pow(2).mean())
            torch.cuda.synchronize()
            for s, fine, crs, crs64, *_ in group:
                fine.close()
                crs.close()
                crs64.close()
        self.params = torch.from_numpy(host_params).to(device)
        torch.cuda.synchronize()
        self.seconds = time.perf_counter() - t0
        self.size = P
        # typical size of the correction: the network's output scale
        self.correction_rms = float((self.target - self.coarse).abs().pow(2).mean().sqrt())
        self.coarse64_rms = float(np.sqrt(sum(float(x) for x in tru_parts) / max(len(tru_parts), 1)))


def train(corr, data, iters, batch, lr=1e-3, seed=SEED, log_every=0):
    """Adam on random minibatches; the step size decays linearly to lr/10.
    The network's output scale is set to the dataset's RMS correction."""
    import torch
    corr.set_output_scale(data.correction_rms)
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        idx = torch.from_numpy(rng.choice(data.size, size=batch, replace=False).astype(np.int32)).cuda()
        step_lr = lr * (1.0 - 0.9 * it / max(1, iters - 1))
        want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
        loss = corr.train_step(data.coarse, data.un, data.target, data.params, idx, step_lr, want_loss=want)
        if want:
            losses.append((it, loss))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def one_step_errors(corr, data, batch=16):
    """Per pair of a (held-out) dataset: the one-step errors
    |C(u_n) - F^8(u_n)| / |F^8(u_n)| and |C(u_n) + N(x_n) - F^8(u_n)| / |F^8(u_n)|
    (relative L2 over the field)."""
    import torch
    coarse_err, corr_err = [], []
    out = torch.empty((batch, data.n, data.n), dtype=torch.complex64, device=data.un.device)
    for b0 in range(0, data.size, batch):
        k = min(batch, data.size - b0)
        corr.apply(data.coarse[b0:b0 + k], data.un[b0:b0 + k], data.params[b0:b0 + k], out[:k])
        for j in range(k):
            t = data.target[b0 + j]
            coarse_err.append(nat.cgl_rel_error(data.coarse[b0 + j], t, nat.CGL_F32)[0])
            corr_err.append(nat.cgl_rel_error(out[j], t, nat.CGL_F32)[0])
    return np.array(coarse_err), np.array(corr_err)


def evaluate(corr, ntraj, seed, n=N, device="cuda", sub=SUB, coarse_steps=COARSE_STEPS):
    """Relative L2 errors at t = coarse_steps * sub * FINE_TAU (4.992 for the
    defaults) of the coarse method with and without the correction against the
    fine method, one held-out trajectory at a time."""
    import torch
    rows = []
    for i in range(ntraj):
        rng = np.random.Generator(np.random.PCG64(seed + 1000 * i))
        par, p, U0 = sample(rng, n)
        prm = torch.tensor([par], dtype=torch.float32, device=device)
        with nat.Plan(p, FINE_TAU, "lawson4", "f64") as fine, nat.Plan(p, FINE_TAU * sub, "lawson4", "f32") as crs:
            uf = nat.to_device(U0, torch.complex128, device)
            fine.step(uf, coarse_steps * sub)
            uc = nat.to_device(U0, torch.complex64, device)
            crs.step(uc, coarse_steps)
            ul = nat.to_device(U0, torch.complex64, device).reshape(1, n, n)
            prev = torch.empty_like(ul)
            for _ in range(coarse_steps):
                prev.copy_(ul)
                crs.step(ul, 1)
                corr.apply(ul, prev, prm, ul)
            torch.cuda.synchronize()
            e_c = nat.cgl_rel_error(uc.to(torch.complex128), uf, nat.CGL_F64)[0]
            e_l = nat.cgl_rel_error(ul.reshape(n, n).to(torch.complex128), uf, nat.CGL_F64)[0]
            rows.append({"params": par, "coarse": e_c, "corrected": e_l})
    return rows
