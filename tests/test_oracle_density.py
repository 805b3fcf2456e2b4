"""Pins of the oracle's density gradient (Eq. gradrhokappa with rho varied
at fixed Vp; CPU).

* Central finite differences of the discrete misfit (Eq. objfwi) along
  random interior density perturbations, 2D and 3D, orders 4 and 8.  The
  edge nodes are left alone: the CPML cells copy them and are held fixed.
* The gradient is the same whether the source field is kept in memory or
  rebuilt from the saved boundaries, and with or without the computing box.
* With a constant impedance change the Vp-Ip chain rule holds:
  dJ/dVp|Ip = dJ/dVp|rho - dJ/drho rho / Vp, checked by finite
  differences along (dVp, -rho dVp / Vp).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S


def _prob(w, **kw):
    args = dict(order=w.order, nb=w.nb, fm=w.fm)
    args.update(kw)
    return O.Problem(w.n, w.d, w.nt, w.dt, **args)


CASES = [
    ("2d_o4", lambda: S.tiny_2d(off_grid=True)),
    ("2d_o8", lambda: S.tiny_2d(order=8, nb=6, off_grid=True, src=(8, 9))),
    ("3d_o4", lambda: S.tiny_3d(off_grid=True, nt=30)),
    ("3d_o8", lambda: S.tiny_3d(order=8, nb=5, off_grid=False, nt=25)),
]


def _observed(prob, w, rng):
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    return 0.8 * seis + 0.05 * np.abs(seis).max() * rng.standard_normal(seis.shape)


def _interior(shape, rng):
    d = np.zeros(shape)
    inner = tuple(slice(1, -1) for _ in shape)
    d[inner] = rng.standard_normal(d[inner].shape)
    return d


def _misfit(prob, w, vp, rho, dobs):
    return O.gradient(prob, vp, rho, w.stf, w.srcs[0], w.recs[0], dobs)[0]


@pytest.mark.parametrize("name,make", CASES)
def test_density_gradient_matches_finite_differences(name, make):
    w = make()
    prob = _prob(w, use_box=False)
    rng = np.random.default_rng(5)
    dobs = _observed(prob, w, rng)
    _, _, _, g = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, with_rho=True)
    rho = w.rho.astype(np.float64)
    dr = _interior(rho.shape, rng)
    eps = 0.05                           # the FD error falls as eps^2: 4e-9 .. 3e-8 here
    fd = (_misfit(prob, w, w.vp, rho + eps * dr, dobs) - _misfit(prob, w, w.vp, rho - eps * dr, dobs)) / (2 * eps)
    an = float(np.sum(g * dr))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_density_gradient_edge_nodes_move_the_cpml():
    """An edge-node perturbation also moves the CPML cells that copy it, so
    finite differences there differ from the gradient, which holds those
    cells fixed: the interior restriction of the pin above is needed."""
    w = S.tiny_2d(off_grid=True)
    prob = _prob(w, use_box=False)
    rng = np.random.default_rng(6)
    dobs = _observed(prob, w, rng)
    _, _, _, g = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, with_rho=True)
    rho = w.rho.astype(np.float64)
    dr = np.zeros_like(rho)
    dr[0, :] = 1.0
    eps = 0.05
    fd = (_misfit(prob, w, w.vp, rho + eps * dr, dobs) - _misfit(prob, w, w.vp, rho - eps * dr, dobs)) / (2 * eps)
    an = float(np.sum(g * dr))
    assert abs(fd - an) > 1e-3 * abs(an)


@pytest.mark.parametrize("name,make", [CASES[1], CASES[3]])
def test_density_gradient_paths_agree(name, make):
    w = make()
    rng = np.random.default_rng(7)
    dobs = _observed(_prob(w), w, rng)
    ref = O.gradient(_prob(w, use_box=False), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, recon=False,
                     with_rho=True)[3]
    for box in (False, True):
        got = O.gradient(_prob(w, use_box=box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, recon=True,
                         with_rho=True)[3]
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


def test_impedance_chain_rule():
    w = S.tiny_2d(order=8, nb=6, off_grid=True, src=(8, 9))
    prob = _prob(w, use_box=False)
    rng = np.random.default_rng(8)
    dobs = _observed(prob, w, rng)
    _, gv, _, gr = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, with_rho=True)
    vp, rho = w.vp.astype(np.float64), w.rho.astype(np.float64)
    ip = vp * rho
    dv = _interior(vp.shape, rng)
    dv[vp >= vp.max()] = 0.0              # keep vmax (and so the CPML profile) fixed
    eps = 1e-2

    def J(e):
        v = vp + e * dv
        return _misfit(prob, w, v, ip / v, dobs)
    fd = (J(eps) - J(-eps)) / (2 * eps)
    an = float(np.sum((gv - gr * rho / vp) * dv))
    assert abs(fd - an) <= 1e-6 * abs(an)
