"""Learned corrector of a coarse exponential step, trained on trajectories of
the fine method (2D periodic cubic CGL, 128 x 128, (-10,10)^2).

  fine   : Lawson4 (eq. lawson4), complex128, tau_f = 0.002   (training target and reference)
  coarse : Lawson4, complex128, tau_c = 0.016 = 8 tau_f
  corrected coarse step: u_{n+1} = C(u_n) + N(x_n)  (cgl_corrector_*)

The network learns the correction delta = F^8(u_n) - C(u_n), formed in FP64
and stored in complex64 (its own size sets its FP32 resolution); the features
are complex64 copies of C(u_n) and u_n, the corrected step adds N(x_n) to the
complex128 coarse result (cgl_corrector_apply_c128).  The correction is the
coarse step's truncation error, about 4e-8 of a state of size 0.2 at this
step: it must not pass through complex64 states, whose resolution is 1e-8.

Parameters per trajectory are drawn from the batched workload's ranges with
a4 = b4 = 0 (cubic): a1 in [0.2,2], b1 in [-2,2], a2 in [0.1,1], a3 in
[-2,-0.5], b3 in [-2,2]; initial data are three random Gaussian bumps.  A
trajectory contributes `snaps` training pairs (u_n, C(u_n), delta) at fine
steps 0, 312, 624, ...  Evaluation runs held-out trajectories to
t = 312 tau_c = 4.992 with and without the correction and compares both with
the fine result.

Every numerical step runs in the library's kernels (plans and corrector);
torch holds device memory, converts between complex128 and complex64 storage
and forms the training targets (a difference of two stored results).
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
    """Device tensors: un, coarse (complex64 copies of u_n and of the
    complex128 coarse result C(u_n)), target = F^sub(u_n) - C(u_n) (formed in
    FP64, stored complex64) [P, n, n], params (float32 [P, 5])."""

    def __init__(self, ntraj, snaps=8, seed=SEED, n=N, device="cuda", concurrency=32, sub=SUB,
                 coarse_steps=COARSE_STEPS):
        """Trajectories run `concurrency` at a time, each on its own CUDA stream
        (one 128^2 instance fills only a few SMs).  The coarse step is `sub`
        fine steps long; snapshots are spread over `coarse_steps` coarse steps."""
        import torch
        P = ntraj * snaps
        self.n = n
        self.un = torch.empty((P, n, n), dtype=torch.complex64, device=device)
        self.coarse = torch.empty_like(self.un)
        self.target = torch.empty_like(self.un)
        host_params = np.empty((P, 5), dtype=np.float32)
        stride = coarse_steps * sub // snaps
        self.sub = sub
        streams = [torch.cuda.Stream() for _ in range(min(concurrency, ntraj))]
        t0 = time.perf_counter()
        for g0 in range(0, ntraj, len(streams)):
            group = []
            for gi, i in enumerate(range(g0, min(ntraj, g0 + len(streams)))):
                s = streams[gi]
                rng = np.random.Generator(np.random.PCG64(seed + 1000 * i))
                par, p, U0 = sample(rng, n)
                fine = nat.Plan(p, FINE_TAU, "lawson4", "f64", stream=s)
                crs = nat.Plan(p, FINE_TAU * sub, "lawson4", "f64", stream=s)
                with torch.cuda.stream(s):
                    u = nat.to_device(U0, torch.complex128, device)
                    v = torch.empty_like(u)
                    w = torch.empty_like(u)
                group.append((s, fine, crs, u, v, w, i))
                host_params[i * snaps:(i + 1) * snaps] = par
            for sn in range(snaps):
                for s, fine, crs, u, v, w, i in group:
                    k = i * snaps + sn
                    with torch.cuda.stream(s):
                        if sn > 0:
                            fine.step(u, stride, stream=s)
                        self.un[k].copy_(u)
                        v.copy_(u)
                        fine.step(v, sub, stream=s)
                        w.copy_(u)
                        crs.step(w, 1, stream=s)
                        self.coarse[k].copy_(w)
                        v.sub_(w)
                        self.target[k].copy_(v)
            torch.cuda.synchronize()
            for s, fine, crs, *_ in group:
                fine.close()
                crs.close()
        self.params = torch.from_numpy(host_params).to(device)
        torch.cuda.synchronize()
        self.seconds = time.perf_counter() - t0
        self.size = P
        # typical size of the correction (the network's output scale), and
        # of the correction relative to the RMS coarse increment of its pair
        # (the output scale of the per-sample mode)
        self.correction_rms = float(self.target.abs().pow(2).mean().sqrt())
        inc = (self.coarse - self.un).abs().pow(2).mean(dim=(1, 2)).sqrt()
        rel = self.target.abs().pow(2).mean(dim=(1, 2)).sqrt() / inc.clamp_min(1e-30)
        self.relative_rms = float(rel.pow(2).mean().sqrt())


def train(corr, data, iters, batch, lr=1e-3, seed=SEED, log_every=0, per_sample=True):
    """Adam on random minibatches, the loss on N(x) - delta (target mode 1);
    the step size decays linearly to lr/10.  per_sample: N is scaled per
    sample by the RMS coarse increment times the dataset's RMS ratio of the
    correction to it (scale mode 1), else by the dataset's RMS correction."""
    import torch
    if per_sample:
        corr.set_scale_mode(1)
        corr.set_output_scale(data.relative_rms)
    else:
        corr.set_scale_mode(0)
        corr.set_output_scale(data.correction_rms)
    corr.set_target_mode(1)
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


def one_step_gains(corr, data, batch=16):
    """Per pair of a (held-out) dataset: ||delta|| / ||N(x_n) - delta||, how
    much the corrected coarse step is closer to the fine step than the coarse
    step alone (1 = no gain)."""
    import torch
    gains = []
    for b0 in range(0, data.size, batch):
        k = min(batch, data.size - b0)
        out = corr.forward(data.coarse[b0:b0 + k], data.un[b0:b0 + k], data.params[b0:b0 + k])
        corr_c = torch.complex(out[:, 0].contiguous(), out[:, 1].contiguous())
        for j in range(k):
            e = nat.cgl_rel_error(corr_c[j].contiguous(), data.target[b0 + j], nat.CGL_F32)[0]
            gains.append(1.0 / e if e > 0 else float("inf"))
    return np.array(gains)


def evaluate(corr, ntraj, seed, n=N, device="cuda", sub=SUB, coarse_steps=COARSE_STEPS):
    """Relative L2 errors at t = coarse_steps * sub * FINE_TAU (4.992 for the
    defaults) of the coarse method with and without the correction against the
    fine method, one held-out trajectory at a time (complex128 states)."""
    import torch
    rows = []
    for i in range(ntraj):
        rng = np.random.Generator(np.random.PCG64(seed + 1000 * i))
        par, p, U0 = sample(rng, n)
        prm = torch.tensor([par], dtype=torch.float32, device=device)
        with nat.Plan(p, FINE_TAU, "lawson4", "f64") as fine, nat.Plan(p, FINE_TAU * sub, "lawson4", "f64") as crs:
            uf = nat.to_device(U0, torch.complex128, device)
            fine.step(uf, coarse_steps * sub)
            uc = nat.to_device(U0, torch.complex128, device)
            crs.step(uc, coarse_steps)
            ul = nat.to_device(U0, torch.complex128, device).reshape(1, n, n)
            prev = torch.empty_like(ul)
            for _ in range(coarse_steps):
                prev.copy_(ul)
                crs.step(ul, 1)
                corr.apply_c128(ul, prev, prm, ul)
            torch.cuda.synchronize()
            e_c = nat.cgl_rel_error(uc, uf, nat.CGL_F64)[0]
            e_l = nat.cgl_rel_error(ul.reshape(n, n), uf, nat.CGL_F64)[0]
            rows.append({"params": par, "coarse": e_c, "corrected": e_l})
    return rows
