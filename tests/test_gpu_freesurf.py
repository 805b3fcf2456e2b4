"""Free surface on the GPU (Sec. 2.1, image method), through the C ABI,
against the FP64 oracle (whose free surface is pinned by the mirrored-domain
identity in tests/test_oracle_freesurf.py).

Sources and receivers straddle the surface (folded interpolation weights),
2D and 3D, orders 4 and 8, box on and off: seismograms, RTM images, the Vp
and density gradients, decimated boundaries, the no-allocation forward
call, and the full-size 3D salt grid.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4
IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def smi():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import smi as mod
    torch.cuda.init()
    return mod


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _gprob(smi, w, **kw):
    return smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, freesurf=True, **kw)


def _oprob(w, **kw):
    return O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm, freesurf=True, **kw)


def _near_surface_2d(order, nt=160):
    w = S.tiny_2d(nz=45, nx=61, nt=nt, order=order, nb=10, src=(0, 30))
    h = w.d[0]
    w.srcs = np.array([[(0.37 if order == 4 else 1.37) * h, 30.2 * h, 0.0]])
    rx = np.arange(2, 59, 4) * h
    w.recs = [np.concatenate([np.stack([np.full(rx.size, z), rx + 0.3 * h, np.zeros(rx.size)], axis=1)
                              for z in (0.0, 0.5 * h, 2.0 * h, 11.0 * h)])]
    return w


def _near_surface_3d(order, nt=60):
    w = S.tiny_3d(nz=28, nx=24, ny=26, nt=nt, nb=8, order=order)
    h = w.d[0]
    w.srcs = np.array([[0.41 * h if order == 4 else 1.41 * h, 11.3 * h, 12.6 * h]])
    w.recs = [np.array([[z, x * h, y * h] for z in (0.0, 0.6 * h, 3.0 * h) for x in (3, 11, 19)
                        for y in (4, 13, 22)])]
    return w


CASES = {
    "2d_o4": lambda: _near_surface_2d(4),
    "2d_o8": lambda: _near_surface_2d(8),
    "3d_o4": lambda: _near_surface_3d(4),
    "3d_o8": lambda: _near_surface_3d(8),
}


@pytest.mark.parametrize("use_box", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_free_surface_seismograms(smi, case, use_box):
    w = CASES[case]()
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w, use_box=use_box), w.srcs, w.recs,
                           _dev(w.stf))[0].cpu().numpy()
    ref = O.forward(_oprob(w, use_box=use_box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    on = np.isclose(w.recs[0][:, 0], 0.0)
    assert np.all(seis[:, on] == 0.0)
    assert _rel(seis, ref) <= SEIS_TOL


@pytest.mark.parametrize("case", sorted(CASES))
def test_free_surface_rtm_and_gradients(smi, case):
    w = CASES[case]()
    rng = np.random.default_rng(12)
    true_rho = w.rho.astype(np.float64) * (1.0 + 0.05 * rng.standard_normal(w.rho.shape))
    dobs = O.forward(_oprob(w), 1.03 * w.vp.astype(np.float64), true_rho, w.stf, w.srcs[0], w.recs[0])
    args = (_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf), _dev(dobs.astype(np.float32)))
    img = smi.smi_rtm(*args)
    _, iref, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), iref) <= IMG_TOL
    J, gv, gr = smi.smi_fwi_gradient_family(*args, family=1)
    Jr, gvr, _, grr = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, with_rho=True)
    e1, e2 = _rel(gv.cpu().numpy(), gvr), _rel(gr.cpu().numpy(), grr)
    print(f"{case}: image {_rel(img.cpu().numpy(), iref):.2e}  dJ/dVp {e1:.2e}  dJ/drho {e2:.2e}")
    assert e1 <= IMG_TOL and e2 <= IMG_TOL
    assert abs(float(J.item()) - Jr) <= 1e-3 * Jr
    assert float(gv[..., 0].abs().max()) == 0.0        # kappa at the surface node acts on nothing


def test_free_surface_decimated_boundaries(smi):
    w = _near_surface_2d(8, nt=400)
    dobs = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w, dr=4), w.srcs, w.recs, _dev(w.stf),
                      _dev(dobs.astype(np.float32)))
    _, ref, _ = O.gradient(_oprob(w, dr=4), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), ref) <= IMG_TOL


@pytest.mark.parametrize("case", ["2d_o8", "3d_o4"])
def test_free_surface_noalloc_matches_forward(smi, case):
    import torch
    w = CASES[case]()
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    prob = _gprob(smi, w)
    a = smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf, flat=True)
    b = torch.empty_like(a)
    smi.smi_forward_noalloc(vp, rho, prob, w.srcs, w.recs, stf, b, flat=True)
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) <= 1e-5


def test_free_surface_salt_3d_full_grid(smi):
    """The 3D salt grid (300^3 + 20 CPML layers, order 8, 150 x 150
    receivers two nodes below the surface), shot 0, first 120 steps."""
    w = S.salt_3d(nt=120).subset([0])
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))[0]
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    plain = O.forward(O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm), w.vp, w.rho, w.stf,
                      w.srcs[0], w.recs[0])
    assert np.linalg.norm(ref - plain) > 0.1 * np.linalg.norm(ref)
    assert _rel(seis.cpu().numpy(), ref) <= SEIS_TOL
