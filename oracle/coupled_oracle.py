"""Plain FP64 CPU oracle for the coupled two-field cubic-quintic CGL system
of Caliari & Cassini (arXiv 2403.02816), Sec. 4.5, eq. (coupled):

    u_t =  a0 d_{x1} u + (a1 + i b1) Lap u + a2 u + (a3 + i b3)|u|^2 u
           + (a4 + i b4)|u|^4 u + a5 |v|^2 u,
    v_t = -a0 d_{x1} v + (a1 + i b1) Lap v + a2 v + (a3 + i b3)|v|^2 v
           + (a4 + i b4)|v|^4 v + a5 |u|^2 v,

periodic in every direction, Fourier pseudospectral in space.  K is block
diagonal (one Kronecker-sum block per field, Sec. 4.5), so every linear flow
acts on u and v separately; the nonlinear part couples them pointwise.

TEST INFRASTRUCTURE ONLY, like ``cgl_oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it; it shares no
code with the CUDA library.  It reuses ``cgl_oracle``'s wavenumbers and error
measures (the same oracle).

State: an array ``W`` of shape ``(2, n_1, ..., n_d)``, ``W[0] = u``,
``W[1] = v``, each indexed like ``cgl_oracle`` grid functions.

Readings where the paper is silent:
- the advection term a0 d_{x1} has the symbol i a0 kappa_1 with the signed
  wavenumbers of ``cgl_oracle.wavenumbers``, except that the Nyquist mode of
  an even n_1 gets 0: that mode is its own mirror image, and only a zero
  first-derivative symbol there keeps the system's symmetry x1 -> L - x1,
  u <-> v on the grid (kappa^2 of the Laplacian is unchanged);
- the nonlinear sub-flow of the splitting schemes is one RK4 step of the
  coupled system W' = g(W) (the paper's choice for the cubic-quintic model,
  Sec. 4.3; the coupled flow has no closed form);
- the schemes are those of Sec. 2 with u replaced by the pair W.

Pins (tests/test_coupled_oracle_pins.py): reduction to ``cgl_oracle`` for
a0 = a5 = 0; exact translation of a Fourier mode under pure advection; the
mirror symmetry (x1 -> L - x1, u <-> v); exact coupled plane waves and the
temporal orders they give.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import cgl_oracle as O


@dataclass
class CoupledProblem:
    """Eq. (coupled) on (lo_1, hi_1) x ... x (lo_d, hi_d), periodic."""

    n: tuple
    lo: tuple
    hi: tuple
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


def symbol(p: CoupledProblem, field: int) -> np.ndarray:
    """Fourier symbol of the linear operator of field 0 (u, advection +a0)
    or 1 (v, advection -a0): (a1 + i b1)(-|kappa|^2) + a2 +- i a0 kappa_1,
    as a full tensor over the grid (Sec. 3.2 with the advection term)."""
    ks = [O.wavenumbers(p.n[mu], p.lo[mu], p.hi[mu]) for mu in range(p.d)]
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = sum(k * k for k in grids)
    k1 = ks[0].copy()
    if p.n[0] % 2 == 0:
        k1[p.n[0] // 2] = 0.0  # first derivative of the Nyquist mode
    K1 = np.meshgrid(k1, *ks[1:], indexing="ij")[0]
    sign = 1.0 if field == 0 else -1.0
    return complex(p.a1, p.b1) * (-k2) + p.a2 + sign * 1j * p.a0 * K1


class CoupledLinear:
    """exp(c tau K) and K for the block-diagonal K (Sec. 4.5)."""

    def __init__(self, prob: CoupledProblem, tau: float):
        self.p = prob
        self.tau = float(tau)
        self.S = [symbol(prob, 0), symbol(prob, 1)]

    def expK(self, W: np.ndarray, c: float) -> np.ndarray:
        """exp(c tau K) W: each field multiplied by exp(c tau S_f) in Fourier
        space (unnormalised forward FFT, 1/N inverse)."""
        return np.stack([np.fft.ifftn(np.exp(c * self.tau * S) * np.fft.fftn(w)) for S, w in zip(self.S, W)])

    def K(self, W: np.ndarray) -> np.ndarray:
        return np.stack([np.fft.ifftn(S * np.fft.fftn(w)) for S, w in zip(self.S, W)])


def g(p: CoupledProblem, W: np.ndarray) -> np.ndarray:
    """The nonlinear part of eq. (coupled) for both fields."""
    u, v = W
    ru = (u * np.conj(u)).real
    rv = (v * np.conj(v)).real
    cu = complex(p.a3, p.b3) * ru + complex(p.a4, p.b4) * ru * ru + p.a5 * rv
    cv = complex(p.a3, p.b3) * rv + complex(p.a4, p.b4) * rv * rv + p.a5 * ru
    return np.stack([cu * u, cv * v])


def nonlinear_flow(p: CoupledProblem, W: np.ndarray, t: float) -> np.ndarray:
    """phi_t: one classical RK4 step of W' = g(W) over time t."""
    k1 = g(p, W)
    k2 = g(p, W + 0.5 * t * k1)
    k3 = g(p, W + 0.5 * t * k2)
    k4 = g(p, W + t * k3)
    return W + (t / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


# --------------------------------------------------------------------------
# Schemes (Sec. 2) on the pair W
# --------------------------------------------------------------------------

def step_strang(L: CoupledLinear, W):
    """eq. Strang."""
    p, tau = L.p, L.tau
    return nonlinear_flow(p, L.expK(nonlinear_flow(p, W, tau / 2), 1.0), tau / 2)


def step_split4(L: CoupledLinear, W):
    """eq. Richardson, explicit form: 4/3 of two half Strang steps (the
    middle half-flows as one flow of tau/2) minus 1/3 of a full one."""
    p, tau = L.p, L.tau
    phi = lambda X, t: nonlinear_flow(p, X, t)
    wn2 = phi(L.expK(phi(W, tau / 2), 1.0), tau / 2)
    v = phi(L.expK(phi(W, tau / 4), 0.5), tau / 2)
    return (4.0 / 3.0) * phi(L.expK(v, 0.5), tau / 4) - (1.0 / 3.0) * wn2


def step_lawson4(L: CoupledLinear, W):
    """eq. lawson4 (if4), all exponential actions as printed."""
    p, tau = L.p, L.tau
    gn = g(p, W)
    un2 = L.expK(W + (tau / 2) * gn, 0.5)
    gn2 = g(p, un2)
    un3 = L.expK(W, 0.5) + (tau / 2) * gn2
    gn3 = g(p, un3)
    un4 = L.expK(W, 1.0) + tau * L.expK(gn3, 0.5)
    gn4 = g(p, un4)
    return L.expK(W + (tau / 6) * gn, 1.0) + (tau / 3) * L.expK(gn2 + gn3, 0.5) + (tau / 6) * gn4


def step_lawson2(L: CoupledLinear, W):
    """eq. lawson2b (if2)."""
    p, tau = L.p, L.tau
    gn = g(p, W)
    un2 = L.expK(W + tau * gn, 1.0)
    return L.expK(W + (tau / 2) * gn, 1.0) + (tau / 2) * g(p, un2)


def step_rk4(L: CoupledLinear, W):
    """eq. RK4 on W' = K W + g(W)."""
    p, tau = L.p, L.tau
    f = lambda X: L.K(X) + g(p, X)
    f1 = f(W)
    f2 = f(W + (tau / 2) * f1)
    f3 = f(W + (tau / 2) * f2)
    f4 = f(W + tau * f3)
    return W + (tau / 6) * (f1 + 2 * f2 + 2 * f3 + f4)


def step_rk2(L: CoupledLinear, W):
    """eq. RK2 (Heun)."""
    p, tau = L.p, L.tau
    f = lambda X: L.K(X) + g(p, X)
    f1 = f(W)
    f2 = f(W + tau * f1)
    return W + (tau / 2) * (f1 + f2)


SCHEMES = {"strang": step_strang, "split4": step_split4, "lawson4": step_lawson4, "lawson2": step_lawson2,
           "rk4": step_rk4, "rk2": step_rk2}
ORDERS = {"strang": 2, "split4": 4, "lawson4": 4, "lawson2": 2, "rk4": 4, "rk2": 2}


def integrate(prob: CoupledProblem, W0: np.ndarray, tau: float, nsteps: int, scheme: str) -> np.ndarray:
    """``nsteps`` constant steps of ``scheme`` from W0 (shape (2, n_1..n_d))."""
    L = CoupledLinear(prob, tau)
    step = SCHEMES[scheme]
    W = np.array(W0, dtype=complex)
    for _ in range(int(nsteps)):
        W = step(L, W)
    return W
