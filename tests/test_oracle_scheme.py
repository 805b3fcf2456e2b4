"""Pins of the oracle's discrete scheme against closed forms (CPU only).

* FD coefficients: exact rationals and polynomial exactness (Sec. 2.1).
* Interior update, staggering and time stepping: the periodic discrete
  plane-wave eigenmode sin(w dt/2) = (dt/2) c |k~| holds to roundoff.
* CFL (Eq. cfl): the oracle's acceptance limit equals the von Neumann limit
  of the fastest (checkerboard) mode.
"""
from fractions import Fraction
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd_coeffs.txt")


def _golden_coeffs():
    table = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        order, l, p, q = map(int, line.split())
        table.setdefault(order, {})[l] = Fraction(p, q)
    return table


@pytest.mark.parametrize("order", [2, 4, 8])
def test_fd_coeffs_match_exact_rationals(order):
    gold = _golden_coeffs()[order]
    a = O.fd_coeffs(order // 2)
    for l, frac in gold.items():
        assert abs(a[l - 1] - float(frac)) <= 4e-16 * max(1.0, abs(float(frac)))


@pytest.mark.parametrize("order", [4, 8])
def test_fd_coeffs_exact_on_polynomials(order):
    """The staggered derivative is exact for x^m, m <= 2N-1, and not for 2N+1."""
    N = order // 2
    a = O.fd_coeffs(N)
    h = 0.37
    x = 1.3
    for m in range(1, 2 * N + 2, 2):
        s = sum(a[l - 1] * ((x + (2 * l - 1) * h / 2) ** m - (x - (2 * l - 1) * h / 2) ** m)
                for l in range(1, N + 1)) / h
        exact = m * x ** (m - 1)
        if m <= 2 * N - 1:
            assert abs(s - exact) <= 1e-12 * max(1.0, abs(exact))
        else:
            assert abs(s - exact) > 1e-6


def _ktilde(a, k, h):
    l = np.arange(1, len(a) + 1)
    return (2.0 / h) * np.sum(a * np.sin((2 * l - 1) * k * h / 2))


def _standing_wave(n, h, modes, c, rho, dt, a):
    """Exact discrete standing wave p^n = cos(w n dt) prod_a cos(k_a x_a) and the
    matching v^{-1/2}; returns (state dict, omega, p(nsteps) function)."""
    ndim = len(n)
    ks = [2 * np.pi * m / (nn * h) for m, nn in zip(modes, n)]
    kt = [_ktilde(a, k, h) for k in ks]
    s = dt / 2 * c * np.sqrt(np.sum(np.square(kt)))
    assert s < 1
    om = 2 / dt * np.arcsin(s)
    coords = np.meshgrid(*[np.arange(nn) * h for nn in reversed(n)], indexing="ij")
    coords = list(reversed(coords))        # coords[a] varies along axis a
    cosk = [np.cos(k * x) for k, x in zip(ks, coords)]
    sink_half = [np.sin(k * (x + h / 2)) for k, x in zip(ks, coords)]
    state = {"p": np.ascontiguousarray(np.prod(cosk, axis=0))}
    names = ["vz", "vx", "vy"]
    for ax in range(ndim):
        V = dt * (1.0 / rho) * kt[ax] / (2 * np.sin(om * dt / 2))
        f = V * np.sin(-om * dt / 2) * sink_half[ax]
        for b in range(ndim):
            if b != ax:
                f = f * cosk[b]
        state[names[ax]] = np.ascontiguousarray(f)
    p0 = state["p"].copy()
    return state, om, (lambda m: np.cos(om * m * dt) * p0)


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("n,modes", [((32, 24), (3, 2)), ((16, 12, 10), (2, 1, 3))])
def test_periodic_plane_wave_eigenmode(order, n, modes):
    h, c, rho, dt = 10.0, 2000.0, 1000.0, 1e-3
    a = O.fd_coeffs(order // 2)
    prob = O.Problem(n, (h,) * len(n), 10, dt, order=order, nb=0, fm=0.0, periodic=True,
                     use_box=False)
    vp = np.full(tuple(reversed(n)), c)
    rh = np.full(vp.shape, rho)
    state, om, exact = _standing_wave(n, h, modes, c, rho, dt, a)
    steps = 60
    O.propagate(prob, vp, rh, state, steps)
    assert np.abs(state["p"] - exact(steps)).max() <= 1e-12


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("ndim", [2, 3])
def test_cfl_limit_is_von_neumann_limit(order, ndim):
    """Eq. cfl accepts exactly the time steps for which the checkerboard mode
    k = pi/h on every axis has |sin(w dt/2)| <= 1."""
    h, c = 10.0, 3000.0
    N = order // 2
    a = O.fd_coeffs(N)
    kt = _ktilde(a, np.pi / h, h)
    dt_vn = 2.0 / (c * np.sqrt(ndim) * kt)      # (dt/2) c sqrt(ndim) kt = 1
    n = (12,) * ndim
    vp = np.full(n, c)
    rho = np.full(n, 1000.0)

    def rc(dt):
        return O.check(O.Problem(n, (h,) * ndim, 10, dt, order=order, nb=4, fm=0.0), vp, rho)

    assert rc(dt_vn * (1 - 1e-9)) == 0
    assert rc(dt_vn * (1 + 1e-9)) == -2


def test_checkerboard_mode_bounded_below_cfl():
    """Just under the limit the fastest mode oscillates without growth."""
    n, h, c, rho = (16, 16), 10.0, 3000.0, 1000.0
    a = O.fd_coeffs(4)
    kt = _ktilde(a, np.pi / h, h)
    dt = 0.999 * 2.0 / (c * np.sqrt(2) * kt)
    prob = O.Problem(n, (h, h), 10, dt, order=8, nb=0, fm=0.0, periodic=True, use_box=False)
    vp = np.full(n, c)
    rh = np.full(n, rho)
    state, om, exact = _standing_wave(n, h, (8, 8), c, rho, dt, a)
    O.propagate(prob, vp, rh, state, 400)
    assert np.abs(state["p"] - exact(400)).max() <= 1e-9
