"""Pins of the coupled-system oracle (Sec. 4.5, eq. coupled) to things other
than itself: the already-pinned single-field oracle in the decoupled case,
the exact translation of a Fourier mode under pure advection, the mirror
symmetry of the system, and exact coupled plane waves with the temporal
orders they give."""
import numpy as np
import pytest

from oracle import cgl_oracle as O
from oracle import coupled_oracle as C

SCHEMES = ["strang", "split4", "lawson4", "lawson2", "rk4", "rk2"]


def grid(p):
    xs = [p.lo[mu] + (p.hi[mu] - p.lo[mu]) * np.arange(p.n[mu]) / p.n[mu] for mu in range(p.d)]
    return np.meshgrid(*xs, indexing="ij")


def smooth_pair(p, rng):
    X = grid(p)
    L = [p.hi[mu] - p.lo[mu] for mu in range(p.d)]
    u = 0.6 * np.exp(1j * 2 * np.pi * X[0] / L[0]) + 0.3 * np.cos(2 * np.pi * X[1] / L[1])
    v = 0.5 * np.exp(-1j * 2 * np.pi * X[1] / L[1]) + 0.2j * np.sin(2 * np.pi * X[0] / L[0])
    return np.stack([u, v]) * (1 + 0.05 * rng.standard_normal(u.shape))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_decoupled_case_reduces_to_the_single_field_oracle(scheme):
    """a0 = a5 = 0: u and v each follow eq. (1), integrated by cgl_oracle."""
    rng = np.random.default_rng(1)
    p = C.CoupledProblem((8, 6), (0.0, 0.0), (7.0, 3.5), 0.0, 0.3, 0.5, -0.2, 1.0, 0.8, -0.1, -0.6, 0.0)
    W0 = smooth_pair(p, rng)
    got = C.integrate(p, W0, 0.01, 5, scheme)
    single = O.OracleProblem(p.n, (O.PERIODIC,) * 2, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)
    if scheme in ("strang", "split4"):
        # the single-field oracle uses the same RK4 flow for cubic-quintic
        assert not single.cubic
    for f in range(2):
        ref = O.integrate(single, W0[f], 0.01, 5, scheme)
        assert O.rel_l2(got[f], ref) < 1e-13


@pytest.mark.parametrize("scheme", ["strang", "split4", "lawson4", "lawson2"])
def test_pure_advection_translates_a_fourier_mode(scheme):
    """a1 = b1 = a2 = 0 and no nonlinearity: u_t = a0 u_x1 moves u0(x1) to
    u0(x1 + a0 t), v to v0(x1 - a0 t); an exponential scheme is exact."""
    p = C.CoupledProblem((16, 4), (0.0, 0.0), (10.0, 2.0), -0.4, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    X = grid(p)
    k = 2 * np.pi * 3 / 10.0
    W0 = np.stack([np.exp(1j * k * X[0]), 2.0 * np.exp(-2j * k * X[0])])
    T, nsteps = 0.7, 7
    got = C.integrate(p, W0, T / nsteps, nsteps, scheme)
    exact = np.stack([np.exp(1j * k * (X[0] + p.a0 * T)), 2.0 * np.exp(-2j * k * (X[0] - p.a0 * T))])
    assert np.max(np.abs(got - exact)) < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES)
def test_mirror_symmetry(scheme):
    """x1 -> L - x1 maps the u equation onto the v equation (the advection
    sign flips): v0(x) = u0(mirror x) keeps v(t) = u(t, mirror x)."""
    rng = np.random.default_rng(5)
    p = C.CoupledProblem((10, 4), (0.0, 0.0), (7.0, 2.0), -0.4, 0.125, 0.5, -0.9, 1.0, 0.8, -0.1, -0.6, 0.5)
    u0 = smooth_pair(p, rng)[0]
    mirror = lambda a: np.roll(a[::-1, :], 1, axis=0)  # index j -> (-j) mod n1
    W0 = np.stack([u0, mirror(u0)])
    got = C.integrate(p, W0, 0.01, 4, scheme)
    assert np.max(np.abs(got[1] - mirror(got[0]))) < 1e-13 * np.max(np.abs(got))
    # and the coupling is really active
    assert np.max(np.abs(got[0] - C.integrate(
        C.CoupledProblem(p.n, p.lo, p.hi, p.a0, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4, 0.0),
        W0, 0.01, 4, scheme)[0])) > 1e-6


def plane_wave_problem():
    """u = a exp(i(k.x - w t)), v = a exp(i(k'.x - w t)), k' = (-k1, k2):
    with a2 = a1|k|^2 - (a3 + a5) a^2 - a4 a^4 the real parts cancel and
    u_t = i (a0 k1 - b1 |k|^2 + b3 a^2 + b4 a^4) u; v likewise (mirror)."""
    n, L = (16, 8), (8.0, 4.0)
    k = np.array([2 * np.pi * 2 / L[0], 2 * np.pi * 1 / L[1]])
    a, a0, a1, b1, a3, b3, a4, b4, a5 = 0.7, -0.4, 0.125, 0.5, 1.0, 0.8, -0.1, -0.6, 0.5
    a2 = a1 * (k @ k) - (a3 + a5) * a * a - a4 * a ** 4
    p = C.CoupledProblem(n, (0.0, 0.0), L, a0, a1, b1, a2, a3, b3, a4, b4, a5)
    lam = a0 * k[0] - b1 * (k @ k) + b3 * a * a + b4 * a ** 4
    X = grid(p)

    def exact(t):
        return np.stack([a * np.exp(1j * (k[0] * X[0] + k[1] * X[1] + lam * t)),
                         a * np.exp(1j * (-k[0] * X[0] + k[1] * X[1] + lam * t))])
    return p, exact


def test_plane_wave_solves_the_system():
    """The residual of eq. (coupled) on the plane wave vanishes (K W + g(W)
    against dW/dt = i lam W), checked on the grid with the oracle's K and g."""
    p, exact = plane_wave_problem()
    W = exact(0.0)
    L = C.CoupledLinear(p, 1.0)
    dWdt = (exact(1e-6) - exact(-1e-6)) / 2e-6
    assert np.max(np.abs(L.K(W) + C.g(p, W) - dWdt)) < 1e-7


@pytest.mark.parametrize("scheme", SCHEMES)
def test_plane_wave_temporal_orders(scheme):
    """Exact solution, no spatial error: the observed order between 20 and 40
    steps to T = 0.2 is the scheme's printed order (2 or 4)."""
    p, exact = plane_wave_problem()
    T = 0.2
    errs = []
    for m in (20, 40):
        W = C.integrate(p, exact(0.0), T / m, m, scheme)
        errs.append(O.rel_l2(W, exact(T)))
    order = O.observed_order(20, errs[0], 40, errs[1])
    assert abs(order - C.ORDERS[scheme]) < 0.15, (scheme, errs, order)
