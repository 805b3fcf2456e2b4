"""Decimated boundary saving in the oracle (Sec. 4.2): the band of every
dr-th step is stored and interpolated in time (Kaiser-windowed sinc, radius
8 samples, shape 8) during source-field reconstruction.

Pins:
- the time interpolator against closed-form sinusoids below the Nyquist
  rate that the paper's dr rule admits;
- the reconstruction against the forward field itself;
- the dr rule (dr <= 5 vmax / vmin);
- the gradient with decimation against the exact (dr = 1) gradient.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

TIME_R, TIME_B = 8, 8.0


@pytest.mark.parametrize("f", [0.02, 0.05, 0.1, 0.2, 0.3])
def test_time_interpolator_reproduces_sinusoids(f):
    """f in cycles per stored sample; 0.3 is about where the dr rule puts the
    top of a Ricker band (2.5 fm) at the largest admitted dr."""
    worst = 0.0
    for x0 in np.linspace(0.0, 1.0, 21) + 40.0:
        first, w = O.kaiser_1d(x0, TIME_R, TIME_B)
        k = first + np.arange(2 * TIME_R)
        got = float(np.sum(w * np.sin(2 * np.pi * f * k + 0.3)))
        worst = max(worst, abs(got - np.sin(2 * np.pi * f * x0 + 0.3)))
    assert worst <= 2e-4


def test_time_interpolator_is_exact_on_stored_samples():
    for x0 in [0.0, 3.0, 17.0]:
        first, w = O.kaiser_1d(x0, TIME_R, TIME_B)
        k = first + np.arange(2 * TIME_R)
        assert np.all(w[k != x0] == 0.0) and w[k == x0][0] == 1.0


def _case():
    return S.layered_fault_2d(nz=60, nx=120, nt=700, nshot=1, order=8)


def _prob(w, dr):
    return O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm, dr=dr)


@pytest.fixture(scope="module")
def fault():
    w = _case()
    seis, snaps = O.forward(_prob(w, 1), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    return w, seis, snaps


def _recon_error(w, snaps, dr):
    rec = O.reconstruct(_prob(w, dr), w.vp, w.rho, w.stf, w.srcs[0])
    # rec[it] = p^{it}; snaps[it] = p^{it+1}
    ref, got = snaps[:-1], rec[1:]
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_reconstruction_with_decimated_boundaries(fault):
    """dr = 1 is the exact reversal; dr = 2, 4 (the rule admits 5 here) stay
    within the interpolator's error times the reconstruction's gain, and the
    error grows with dr."""
    w, seis, snaps = fault
    e1 = _recon_error(w, snaps, 1)
    e2 = _recon_error(w, snaps, 2)
    e4 = _recon_error(w, snaps, 4)
    assert e1 <= 1e-10
    assert 1e-9 < e2 < e4 <= 1e-4


def test_dr_rule_rejects_aliasing_ratios(fault):
    w, _, _ = fault
    ratio = 5.0 * w.vp.max() / w.vp.min()
    assert O.check(_prob(w, int(np.floor(ratio))), w.vp, w.rho) == 0
    assert O.check(_prob(w, int(np.floor(ratio)) + 1), w.vp, w.rho) == -1


def test_gradient_with_decimated_boundaries(fault):
    w, seis, _ = fault
    dobs = O.forward(_prob(w, 1), w.vp_true, w.rho, w.stf, w.srcs[0], w.recs[0])
    J1, g1, _ = O.gradient(_prob(w, 1), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    J4, g4, _ = O.gradient(_prob(w, 4), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert J4 == J1                                   # the forward pass is unchanged
    assert np.linalg.norm(g4 - g1) <= 1e-4 * np.linalg.norm(g1)
