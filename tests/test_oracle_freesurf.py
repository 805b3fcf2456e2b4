"""Pins of the oracle's free surface (Sec. 2.1: image method on the top face,
antisymmetric pressure, symmetric vertical velocity; CPU).

* Image method: with the free surface, the field below the surface equals
  the field of the same source plus a negated image source in a model
  mirrored about the surface node, computed without a free surface (both
  faces absorbing); exact for the discrete scheme, so to FP64 rounding.
  Sources and receivers straddle the surface, so the folded interpolation
  weights are covered.
* Pressure at the surface node is zero: a receiver there records nothing.
* Adjoint: the dot-product identity with the free surface (box off and on).
* Gradient: central finite differences of the misfit for Vp and rho.
* Reconstruction: the source field rebuilt from the saved boundaries equals
  the stored field, and the gradient is the same either way.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S


def _prob(w, **kw):
    args = dict(order=w.order, nb=w.nb, fm=w.fm)
    args.update(kw)
    return O.Problem(w.n, w.d, w.nt, w.dt, **args)


def _near_surface_2d(order):
    w = S.tiny_2d(nz=26, nx=22, nt=90, order=order, nb=6 if order == 8 else 5, src=(0, 9))
    h = w.d[0]
    w.srcs = np.array([[0.37 * h if order == 4 else 1.37 * h, 9.2 * h, 0.0]])
    rx = np.arange(2, 20, 3) * h
    w.recs = [np.concatenate([np.stack([np.full(rx.size, z), rx + 0.3 * h, np.zeros(rx.size)], axis=1)
                              for z in (0.0, 0.5 * h, 2.0 * h, 7.0 * h)])]
    return w


def _near_surface_3d():
    w = S.tiny_3d(nz=14, nx=12, ny=11, nt=40, nb=5)
    h = w.d[0]
    w.srcs = np.array([[0.41 * h, 5.3 * h, 4.6 * h]])
    w.recs = [np.array([[z, x * h, y * h] for z in (0.0, 0.6 * h, 3.0 * h) for x in (2, 6) for y in (3, 7)])]
    return w


CASES = [
    ("2d_o4", lambda: _near_surface_2d(4)),
    ("2d_o8", lambda: _near_surface_2d(8)),
    ("3d_o4", _near_surface_3d),
]


def _mirror(a, nz):
    """Model mirrored about the first z node: k' = k + nz - 1 <-> k and
    nz - 1 - k (z is the last numpy axis)."""
    return np.concatenate([a[..., :0:-1], a], axis=-1)


def _shift(pts, dz):
    p = np.array(pts, dtype=np.float64).copy()
    p[:, 0] += dz
    return p


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("use_box", [False, True])
def test_image_method_equals_mirrored_domain(name, make, use_box):
    w = make()
    nz = w.n[0]
    top = (nz - 1) * w.d[0]
    got = O.forward(_prob(w, freesurf=True, use_box=use_box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    big = O.Problem((2 * nz - 1,) + tuple(w.n[1:]), w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm,
                    use_box=False)
    vp2, rho2 = _mirror(w.vp, nz), _mirror(w.rho, nz)
    rec2 = _shift(w.recs[0], top)
    src = _shift(w.srcs, top)[0]
    img = src.copy()
    img[0] = top - w.srcs[0][0]
    ref = (O.forward(big, vp2, rho2, w.stf, src, rec2) - O.forward(big, vp2, rho2, w.stf, img, rec2))
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # and the free surface matters: without it the records differ at O(1)
    plain = O.forward(_prob(w, use_box=use_box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(plain - got) > 0.1 * np.linalg.norm(got)


@pytest.mark.parametrize("name,make", CASES)
def test_surface_receivers_record_zero(name, make):
    w = make()
    seis = O.forward(_prob(w, freesurf=True), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    on = np.isclose(w.recs[0][:, 0], 0.0)
    assert on.any() and np.all(seis[:, on] == 0.0)
    assert np.abs(seis[:, ~on]).max() > 0


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("box_mode", [0, 1])
def test_dot_product_identity_with_free_surface(name, make, box_mode):
    w = make()
    prob = _prob(w, freesurf=True, use_box=bool(box_mode))
    rng = np.random.default_rng(1)
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    d = rng.standard_normal(seis.shape)
    sbar = O.adjoint(prob, w.vp, w.rho, w.srcs[0], w.recs[0], d, box_mode=box_mode)
    lhs = float(np.sum(seis * d))
    rhs = float(np.sum(w.stf.astype(np.float64) * sbar))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _observed(prob, w, rng):
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    return 0.8 * seis + 0.05 * np.abs(seis).max() * rng.standard_normal(seis.shape)


def _interior(shape, rng):
    d = np.zeros(shape)
    inner = tuple(slice(1, -1) for _ in shape)
    d[inner] = rng.standard_normal(d[inner].shape)
    return d


@pytest.mark.parametrize("name,make", CASES[:2])
def test_free_surface_gradients_match_finite_differences(name, make):
    w = make()
    prob = _prob(w, freesurf=True, use_box=False)
    rng = np.random.default_rng(3)
    dobs = _observed(prob, w, rng)
    _, gv, _, gr = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, with_rho=True)
    vp, rho = w.vp.astype(np.float64), w.rho.astype(np.float64)
    J = lambda v, r: O.gradient(prob, v, r, w.stf, w.srcs[0], w.recs[0], dobs)[0]
    dm = _interior(vp.shape, rng)
    dm[vp >= vp.max()] = 0.0          # keep vmax (and so the CPML profile) fixed
    assert np.all(gv[..., 0] == 0.0)  # kappa at the surface node acts on nothing (p = 0 there)
    eps = 1e-3
    fd = (J(vp + eps * dm, rho) - J(vp - eps * dm, rho)) / (2 * eps)
    assert abs(fd - float(np.sum(gv * dm))) <= 1e-6 * abs(fd)
    dr = _interior(rho.shape, rng)
    eps = 0.05
    fd = (J(vp, rho + eps * dr) - J(vp, rho - eps * dr)) / (2 * eps)
    assert abs(fd - float(np.sum(gr * dr))) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("use_box", [False, True])
def test_reconstruction_with_free_surface(name, make, use_box):
    w = make()
    prob = _prob(w, freesurf=True, use_box=use_box)
    _, snap = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    rec = O.reconstruct(prob, w.vp, w.rho, w.stf, w.srcs[0])
    assert np.abs(rec[1:] - snap[:-1]).max() <= 1e-10 * np.abs(snap).max()
    rng = np.random.default_rng(4)
    dobs = _observed(prob, w, rng)
    for mode in ("fwi", "rtm"):
        g1 = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode=mode, recon=True)[1]
        g0 = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode=mode, recon=False)[1]
        assert np.abs(g1 - g0).max() <= 1e-10 * np.abs(g0).max()


def test_free_surface_needs_room_for_the_image():
    w = _near_surface_2d(8)
    assert O.check(_prob(w, freesurf=True, nb=3), w.vp, w.rho) == -1


def test_decimated_reconstruction_with_free_surface():
    """Decimated boundaries (Sec. 4.2) with the free surface: dr = 1 is the
    exact reversal; dr = 2 and 4 stay within the interpolator's error, which
    grows with dr (the image half nodes are part of the top band)."""
    w = S.layered_fault_2d(nz=60, nx=120, nt=700, nshot=1, order=8)
    errs = {}
    for dr in (1, 2, 4):
        prob = _prob(w, freesurf=True, dr=dr)
        _, snap = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
        rec = O.reconstruct(prob, w.vp, w.rho, w.stf, w.srcs[0])
        errs[dr] = np.linalg.norm(rec[1:] - snap[:-1]) / np.linalg.norm(snap[:-1])
    assert errs[1] <= 1e-10
    assert 1e-9 < errs[2] < errs[4] <= 1e-4
