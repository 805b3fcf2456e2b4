"""Physics pins of the oracle (CPU only).

* Source scaling and timing: analytic homogeneous Green's functions,
  3D p = s'(t - r/c) / (4 pi c^2 r) and 2D p = (1/(2 pi c^2)) int_0^inf
  s'(t - (r/c) cosh u) du, for f_p = s(t) delta(x) in Eq. acoustic; the
  injection p += dt s(it dt) w / dV samples the source half a step before
  its nominal time (n+1/2) dt, so the analytic trace is delayed by dt/2.
* CPML (Sec. 2.1): reflections from the 20-layer CPML are orders of
  magnitude below those of an unabsorbing edge, measured against a grid so
  large that its edges are never reached.
* Computing box (Sec. 4.1): monotone growth at the wave speed, and a
  truncation that changes nothing measurable (fields outside it are zero
  to roundoff in an unboxed run).
* Kaiser-windowed sinc (Hicks 2002, Sec. 2.1): exact delta on nodes, I0
  against scipy's, interpolation of a smooth field.
* Setup checks (Sec. 3.8): CFL, dispersion and geometry errors.
"""
import numpy as np
import pytest
from scipy import special

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S


def _ricker_dot(t, fm, t0):
    tau = t - t0
    a = (np.pi * fm * tau) ** 2
    dadt = 2.0 * np.pi ** 2 * fm ** 2 * tau
    return (-2.0 * dadt - (1.0 - 2.0 * a) * dadt) * np.exp(-a)


def test_green_function_2d():
    c, h, fm, dt, nt = 2000.0, 10.0, 10.0, 1e-3, 520
    n = (161, 161)
    vp = np.full(n, c, np.float32)
    rho = np.full(n, 1000.0, np.float32)
    prob = O.Problem(n, (h, h), nt, dt, order=8, nb=20, fm=fm)
    stf = S.ricker(nt, dt, fm)
    src = np.array([80 * h, 80 * h, 0.0])
    rec = np.array([[80 * h, (80 + k) * h, 0.0] for k in (60, 75)] + [[15 * h, 80 * h, 0.0]])
    seis = O.forward(prob, vp, rho, stf, src, rec)
    t = (np.arange(nt) + 1) * dt
    u = np.linspace(0.0, 8.0, 20001)
    for j, r in enumerate(rec):
        rr = np.hypot(*(r - src)[:2])
        ana = np.array([np.trapezoid(_ricker_dot(tt - dt / 2 - rr / c * np.cosh(u), fm, 1.2 / fm), u)
                        for tt in t]) / (2 * np.pi * c * c)
        err = np.linalg.norm(seis[:, j] - ana) / np.linalg.norm(ana)
        assert err < 0.02, (rr, err)


def test_green_function_3d():
    c, h, fm, dt, nt = 2000.0, 10.0, 12.0, 1e-3, 400
    n = (80, 28, 28)
    vp = np.full(tuple(reversed(n)), c, np.float32)
    rho = np.full(vp.shape, 1000.0, np.float32)
    prob = O.Problem(n, (h, h, h), nt, dt, order=8, nb=10, fm=fm)
    stf = S.ricker(nt, dt, fm)
    src = np.array([14 * h, 14 * h, 14 * h])
    rec = np.array([[(14 + k) * h, 14 * h, 14 * h] for k in (45, 55)])
    seis = O.forward(prob, vp, rho, stf, src, rec)
    t = (np.arange(nt) + 1) * dt
    for j, r in enumerate(rec):
        rr = np.linalg.norm(r - src)
        ana = _ricker_dot(t - dt / 2 - rr / c, fm, 1.2 / fm) / (4 * np.pi * c * c * rr)
        err = np.linalg.norm(seis[:, j] - ana) / np.linalg.norm(ana)
        assert err < 0.025, (rr, err)


def test_cpml_absorbs():
    c, h, dt, nt, fm = 2000.0, 10.0, 1e-3, 900, 10.0
    vp = np.full((101, 101), c, np.float32)
    rho = np.full(vp.shape, 1000.0, np.float32)
    src = np.array([500.0, 500.0, 0.0])
    rec = np.array([[500.0, 500.0 + 10.0 * k, 0.0] for k in range(-40, 41, 10)])
    stf = S.ricker(nt, dt, fm)
    small = O.Problem((101, 101), (h, h), nt, dt, order=8, nb=20, fm=fm)
    big = O.Problem((501, 501), (h, h), nt, dt, order=8, nb=20, fm=fm)
    vb = np.full((501, 501), c, np.float32)
    shift = np.array([2000.0, 2000.0, 0.0])
    ref = O.forward(big, vb, np.full(vb.shape, 1000.0, np.float32), stf, src + shift, rec + shift)
    absorbed = O.forward(small, vp, rho, stf, src, rec)
    small.cpml_R = 1.0
    hard = O.forward(small, vp, rho, stf, src, rec)
    e_abs = np.linalg.norm(absorbed - ref) / np.linalg.norm(ref)
    e_hard = np.linalg.norm(hard - ref) / np.linalg.norm(ref)
    assert e_hard > 0.05
    assert e_abs < 1e-3
    assert e_abs < 0.01 * e_hard


def test_cpml_profile_shape():
    """Damping is zero in the physical domain, positive and growing towards
    the outer edge in the layers, with 0 < b < 1."""
    w = S.tiny_2d(nb=8)
    prob = O.Problem(w.n, w.d, w.nt, w.dt, order=4, nb=8, fm=w.fm)
    for vgrid in (0, 1):
        a, b = O.cpml_profile(prob, w.vp, w.rho, axis=0, vgrid=bool(vgrid))
        L, H = 8, 8 + w.n[0] - 1
        inner = slice(L, H) if vgrid else slice(L, H + 1)
        assert np.all(a[inner] == 0) and np.all(b[inner] == 0)
        assert np.all(a[:L] < 0) and np.all((b[:L] > 0) & (b[:L] < 1))
        assert np.all(np.diff(b[:L]) > 0)        # less damping towards the interior


def test_box_is_a_lossless_truncation():
    w = S.two_layer_2d(nt=500)
    prob = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=20, fm=w.fm, use_box=False)
    s_off, snap = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    prob.use_box = True
    s_on = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(s_on - s_off) <= 1e-12 * np.linalg.norm(s_off)
    lo, hi = O.box_table(prob, w.vp, w.rho, w.srcs[0], 0, w.nt)
    peak = np.abs(snap).max()
    for n in range(0, w.nt, 7):
        outside = np.ones(snap.shape[1:], bool)
        zl, zh = lo[n, 0] - 20, hi[n, 0] - 20
        xl, xh = lo[n, 1] - 20, hi[n, 1] - 20
        outside[max(xl, 0):xh + 1, max(zl, 0):zh + 1] = False
        if outside.any():
            assert np.abs(snap[n][outside]).max() <= 1e-12 * peak


def test_box_grows_monotonically_at_the_wave_speed():
    w = S.random_smooth_3d(nz=40, nx=60, ny=50, nt=400)
    prob = O.Problem(w.n, w.d, w.nt, w.dt, order=8, nb=20, fm=w.fm)
    lo, hi = O.box_table(prob, w.vp, w.rho, w.srcs[0], 0, w.nt)
    assert np.all(np.diff(lo, axis=0) <= 0) and np.all(np.diff(hi, axis=0) >= 0)
    # before clipping, the half-width grows by vmax dt / h cells per step
    vmax = float(w.vp.max())
    grow = hi[100, 1] - hi[0, 1]
    assert abs(grow - vmax * w.dt / w.d[1] * 100) <= 1.0
    # the source stencil (plus the two half-step stencils) is inside at n = 0
    src_x = int(round(w.srcs[0][1] / w.d[1])) + 20
    assert lo[0, 1] <= src_x - 8 and hi[0, 1] >= src_x + 8
    # empty box before the first step
    lo1, hi1 = O.box_table(prob, w.vp, w.rho, w.srcs[0], -1, 1)
    assert np.all(hi1 < lo1)


def test_bessel_i0_matches_scipy():
    for x in (0.0, 0.5, 2.0, 4.0, 6.31, 12.0):
        assert abs(O.bessel_i0(x) - special.i0(x)) <= 1e-14 * special.i0(x)


def test_kaiser_sinc_on_node_is_exact_delta():
    for ri in (2, 4):
        first, w = O.kaiser_1d(17.0, ri, 4.0)
        assert first == 17 - ri + 1
        assert w[ri - 1] == 1.0 and np.count_nonzero(w) == 1


@pytest.mark.parametrize("ri", [2, 4])
def test_kaiser_sinc_interpolates_smooth_fields(ri):
    for x0 in (10.25, 10.5, 10.8):
        first, w = O.kaiser_1d(x0, ri, 4.0)
        nodes = first + np.arange(2 * ri)
        assert abs(w.sum() - 1.0) < 0.03
        k = 2 * np.pi / 12.0                     # 12 cells per wavelength
        approx = np.sum(w * np.cos(k * nodes))
        assert abs(approx - np.cos(k * x0)) < 0.02
        if x0 == 10.5:
            assert np.allclose(w, w[::-1], rtol=0, atol=1e-15)


def test_setup_errors():
    w = S.tiny_2d()
    ok = O.Problem(w.n, w.d, w.nt, w.dt, order=4, nb=6, fm=w.fm)
    assert O.check(ok, w.vp, w.rho) == 0
    bad_dt = O.Problem(w.n, w.d, w.nt, 5e-3, order=4, nb=6, fm=w.fm)
    assert O.check(bad_dt, w.vp, w.rho) == -2
    bad_f = O.Problem(w.n, w.d, w.nt, w.dt, order=4, nb=6, fm=40.0)
    assert O.check(bad_f, w.vp, w.rho) == -3
    with pytest.raises(O.OracleError) as e:
        O.forward(ok, w.vp, w.rho, w.stf, np.array([-50.0, 10.0, 0.0]), w.recs[0])
    assert e.value.rc == -1
