"""Pins of the oracle's adjoint, gradient, reconstruction and imaging (CPU).

* Adjoint: the dot-product identity <L f, d> = <f, L^T d> (L: wavelet ->
  seismograms) to FP64 roundoff, with CPML, in 2D and 3D, without the box
  and with the same (forward) box sequence; and L built column by column by
  brute force on a tiny grid.
* Reciprocity: kappa(x_s) p_{s->r} = kappa(x_r) p_{r->s}, exact for the
  leap-frog scheme with zero-padded edges (the one-step map M satisfies
  W M W^-1 = M^T with W = diag(1/kappa, -1/b)).
* Gradient (Eq. gradrhokappa): central finite differences of the discrete
  misfit (Eq. objfwi) along random interior perturbations.
* Reconstruction (Sec. 4.2, dr = 1): the source field rebuilt backwards
  from the saved bands equals the stored forward field.
* RTM image (Eq. rtmimage): equals the cross-correlation computed from a
  receiver field built by brute-force impulse responses.
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


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("box_mode", [0, 1])
def test_dot_product_identity(name, make, box_mode):
    w = make()
    prob = _prob(w, use_box=bool(box_mode))
    rng = np.random.default_rng(1)
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    d = rng.standard_normal(seis.shape)
    sbar = O.adjoint(prob, w.vp, w.rho, w.srcs[0], w.recs[0], d, box_mode=box_mode)
    lhs = float(np.sum(seis * d))
    rhs = float(np.sum(w.stf.astype(np.float64) * sbar))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_equals_brute_force_transpose():
    w = S.tiny_2d(nz=12, nx=10, nt=8, nb=3, src=(5, 4), rec_z=3, rec_step=3, off_grid=True)
    prob = _prob(w, use_box=False)
    nt = w.nt
    cols = []
    for j in range(nt):
        e = np.zeros(nt)
        e[j] = 1.0
        cols.append(O.forward(prob, w.vp, w.rho, e, w.srcs[0], w.recs[0]).ravel())
    L = np.stack(cols, axis=1)                      # (nt*nrec, nt)
    rng = np.random.default_rng(2)
    for _ in range(3):
        d = rng.standard_normal(L.shape[0])
        sbar = O.adjoint(prob, w.vp, w.rho, w.srcs[0], w.recs[0], d)
        assert np.abs(sbar - L.T @ d).max() <= 1e-12 * np.abs(L.T @ d).max()


def _kappa(w, pos):
    idx = tuple(int(round(p / h)) for p, h in zip(pos[:w.ndim], w.d))
    i = tuple(reversed(idx))
    return float(w.rho[i]) * float(w.vp[i]) ** 2


@pytest.mark.parametrize("ndim", [2, 3])
def test_reciprocity_zero_padded(ndim):
    if ndim == 2:
        w = S.tiny_2d(nt=120)
        a, b = np.array([50.0, 90.0, 0.0]), np.array([150.0, 40.0, 0.0])
    else:
        w = S.tiny_3d(nt=60)
        a, b = np.array([40.0, 50.0, 40.0]), np.array([100.0, 20.0, 70.0])
    prob = _prob(w, cpml_R=1.0, use_box=False)
    sab = O.forward(prob, w.vp, w.rho, w.stf, a, b[None])[:, 0]
    sba = O.forward(prob, w.vp, w.rho, w.stf, b, a[None])[:, 0]
    lhs, rhs = _kappa(w, a) * sab, _kappa(w, b) * sba
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


def test_reciprocity_with_cpml_is_approximate():
    """The absorbing layers break exact symmetry; the defect stays small."""
    w = S.tiny_2d(nt=300)
    a, b = np.array([50.0, 90.0, 0.0]), np.array([150.0, 40.0, 0.0])
    prob = _prob(w, use_box=False)
    sab = O.forward(prob, w.vp, w.rho, w.stf, a, b[None])[:, 0]
    sba = O.forward(prob, w.vp, w.rho, w.stf, b, a[None])[:, 0]
    lhs, rhs = _kappa(w, a) * sab, _kappa(w, b) * sba
    rel = np.linalg.norm(lhs - rhs) / np.linalg.norm(lhs)
    assert rel < 5e-2


def _observed(prob, w, rng):
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    return 0.8 * seis + 0.05 * np.abs(seis).max() * rng.standard_normal(seis.shape)


@pytest.mark.parametrize("name,make", CASES)
def test_gradient_matches_finite_differences(name, make):
    w = make()
    prob = _prob(w, use_box=False)
    rng = np.random.default_rng(3)
    dobs = _observed(prob, w, rng)
    J, g, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    vp = w.vp.astype(np.float64)
    dm = np.zeros_like(vp)
    inner = tuple(slice(1, -1) for _ in range(w.ndim))
    dm[inner] = rng.standard_normal(dm[inner].shape)
    dm[vp >= vp.max()] = 0.0          # keep vmax (and so the CPML profile) fixed
    eps = 1e-3
    Jp = O.gradient(prob, vp + eps * dm, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)[0]
    Jm = O.gradient(prob, vp - eps * dm, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)[0]
    fd = (Jp - Jm) / (2 * eps)
    an = float(np.sum(g * dm))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_misfit_is_zero_for_exact_data_and_quadratic_in_residual():
    w = S.tiny_2d()
    prob = _prob(w)
    seis = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    J0, g0, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], seis)
    assert J0 == 0.0 and np.all(g0 == 0.0)
    J1 = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], seis - 1e-6)[0]
    J2 = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], seis - 2e-6)[0]
    assert abs(J1 - 0.5 * seis.size * 1e-12) <= 1e-9 * J1
    assert abs(J2 / J1 - 4.0) <= 1e-9


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("use_box", [False, True])
def test_reconstruction_equals_forward_field(name, make, use_box):
    w = make()
    prob = _prob(w, use_box=use_box)
    _, snap = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    rec = O.reconstruct(prob, w.vp, w.rho, w.stf, w.srcs[0])
    scale = np.abs(snap).max()
    assert np.abs(rec[1:] - snap[:-1]).max() <= 1e-10 * scale     # rec[it] = p^{it}
    assert np.abs(rec[0]).max() == 0.0                             # p^0 = 0


@pytest.mark.parametrize("name,make", CASES[:3])
@pytest.mark.parametrize("mode", ["fwi", "rtm"])
def test_boundary_reconstruction_equals_stored_wavefield(name, make, mode):
    w = make()
    prob = _prob(w)
    rng = np.random.default_rng(4)
    dobs = _observed(prob, w, rng)
    J1, g1, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode=mode,
                           recon=True)
    J0, g0, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode=mode,
                           recon=False)
    assert J1 == J0
    assert np.abs(g1 - g0).max() <= 1e-10 * np.abs(g0).max()


def test_rtm_image_equals_brute_force_crosscorrelation():
    """Receiver field kappa*pbar(it) built from impulse responses: pbar(it)(x)
    = d <seis, d_obs> / d p^{it+1}(x), obtained by propagating a unit
    pressure impulse at x from time level it+1 and recording."""
    w = S.tiny_2d(nz=12, nx=10, nt=10, nb=3, src=(5, 4), rec_z=3, rec_step=3, off_grid=True)
    prob = _prob(w, use_box=False)
    rng = np.random.default_rng(5)
    dobs = rng.standard_normal((w.nt, len(w.recs[0])))
    _, img, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm",
                           recon=False)
    _, snap = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    nb = w.nb
    ext = prob.ext_shape
    # impulse responses G[x][m, r]: record at step it+m of a unit p at level it+1
    # (m = 0 is the record of step it itself)
    brute = np.zeros(prob.shape)
    K = w.rho.astype(np.float64) * w.vp.astype(np.float64) ** 2
    for ix in range(w.n[1]):
        for iz in range(w.n[0]):
            st = {k: np.zeros(ext) for k in ("p", "vz", "vx")}
            st["p"][ix + nb, iz + nb] = 1.0
            g = O.propagate(prob, w.vp, w.rho, st, w.nt, rec=w.recs[0])   # records of steps it+1..
            # record of step it at node x itself: the receiver weights at x
            resp0 = np.array([_rec_weight(prob, r, iz, ix) for r in w.recs[0]])
            for it in range(w.nt):
                pbar = resp0 @ dobs[it]
                for m in range(1, w.nt - it):
                    pbar += g[m - 1] @ dobs[it + m]
                brute[ix, iz] += K[ix, iz] * pbar * snap[it, ix, iz]
    assert np.abs(img - brute).max() <= 1e-10 * np.abs(brute).max()


def _rec_weight(prob, r, iz, ix):
    """Weight of physical node (iz, ix) in the Kaiser-sinc stencil of r."""
    w = 1.0
    for ax, i in ((0, iz), (1, ix)):
        first, wts = O.kaiser_1d(r[ax] / prob.d[ax] + prob.nb, prob.order // 2, prob.kaiser_b)
        j = i + prob.nb - first
        w *= wts[j] if 0 <= j < len(wts) else 0.0
    return w


def test_normalised_image_is_the_image_over_the_forward_illumination():
    """Normalised imaging condition (Sec. 2.3): the oracle's image divided
    by sum_it (p^{it+1})^2 + eps, eps = 1e-3 of its maximum, where the
    illumination here comes from the stored forward snapshots instead of
    the reconstructed source field."""
    w = S.tiny_2d(nz=40, nx=44, nt=120, nb=8, order=8, src=(10, 20))
    prob = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm)
    dobs, snaps = O.forward(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], snapshots=True)
    _, img, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    _, nimg, _ = O.gradient(prob, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm_norm")
    ill = np.sum(snaps ** 2, axis=0)
    ref = img / (ill + 1e-3 * ill.max())
    assert np.linalg.norm(nimg - ref) <= 1e-9 * np.linalg.norm(ref)


def test_gradient_does_not_depend_on_the_thread_count():
    """The parallel adjoint sweep (chunks of the outermost axis in two
    colours) gives the one-thread result up to FP64 rounding order, and a
    one-thread call does not leave later default calls on one thread."""
    w = S.tiny_3d(order=8, nb=5, nt=25)
    seis = O.forward(_prob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    dobs = 0.9 * seis
    default = O.max_threads()
    J1, g1, _ = O.gradient(_prob(w, nthreads=1), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert O.max_threads() == default
    Jn, gn, _ = O.gradient(_prob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert abs(Jn - J1) <= 1e-12 * J1
    assert np.linalg.norm(gn - g1) <= 1e-12 * np.linalg.norm(g1)
