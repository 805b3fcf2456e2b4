"""Decimated boundary saving on the GPU (Sec. 4.2): the boundary of every
dr-th step is stored and interpolated in time during reconstruction.

- **Parity.**  GPU images and gradients match the FP64 oracle run with the
  same dr within the image / gradient bar (1e-3 relative L2).  The
  oracle's decimation is pinned separately (tests/test_oracle_decimation.py).
- **Properties at scale.**  At a workload's largest admitted dr, the image
  stays close to the dr = 1 image, and the call's device footprint shrinks.
- **Errors.**  A ratio above the dr rule is an argument error.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

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
    return smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, **kw)


def _oprob(w, **kw):
    return O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm, **kw)


CASES = {
    # name: (workload, dr); each dr within the rule 5 vmax / vmin of its model
    "2d_o8_dr5": (lambda: S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30)), 5),
    "2d_o4_off_dr7_nobox": (lambda: S.tiny_2d(nz=50, nx=44, nt=150, nb=8, src=(9, 21), off_grid=True), 7),
    "3d_o8_dr3": (lambda: S.tiny_3d(nz=28, nx=24, ny=26, nt=60, nb=8, order=8), 3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_decimated_rtm_image_matches_oracle(smi, case):
    make, dr = CASES[case]
    w = make()
    box = "nobox" not in case
    dobs = O.forward(_oprob(w, use_box=box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w, dr=dr, use_box=box), w.srcs, w.recs,
                      _dev(w.stf), _dev(dobs.astype(np.float32)))
    _, ref, _ = O.gradient(_oprob(w, dr=dr, use_box=box), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs,
                           mode="rtm")
    assert _rel(img.cpu().numpy(), ref) <= IMG_TOL


def test_decimated_fwi_gradient_matches_oracle(smi):
    """Layered-fault 2D model, order 8, 700 steps, dr = 4 (the rule admits 5)."""
    w = S.layered_fault_2d(nz=60, nx=120, nt=700, nshot=1, order=8)
    dobs = O.forward(_oprob(w), w.vp_true, w.rho, w.stf, w.srcs[0], w.recs[0])
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w, dr=4), w.srcs, w.recs,
                                _dev(w.stf), _dev(dobs.astype(np.float32)))
    Jr, gr, _ = O.gradient(_oprob(w, dr=4), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert _rel(g.cpu().numpy(), gr) <= IMG_TOL
    assert abs(float(J.item()) - Jr) <= 1e-3 * Jr


def test_largest_decimation_at_scale(smi):
    """3D salt stand-in at 100^3 (vmax / vmin = 2.25, the rule admits
    dr = 11): the RTM image with dr = 10, the paper's 3D default, stays
    within 1e-3 of the dr = 1 image; the stored boundaries shrink about 10x."""
    import torch
    w = S.salt_3d(n=100, nt=400, nshot=1)
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    gp1, gp10 = _gprob(smi, w), _gprob(smi, w, dr=10)
    dobs = smi.smi_forward(vp, rho, gp1, w.srcs, w.recs, stf)[0].contiguous()
    i1 = smi.smi_rtm(vp, rho, gp1, w.srcs, w.recs, stf, dobs)
    i10 = smi.smi_rtm(vp, rho, gp10, w.srcs, w.recs, stf, dobs)
    err = float(torch.linalg.norm(i10 - i1) / torch.linalg.norm(i1))
    print(f"dr=10 image vs dr=1: {err:.2e}")
    assert err <= 1e-3
    b1 = smi.smi_query(vp, rho, gp1, w.srcs, w.recs, stf, kind="rtm")[2]
    b10 = smi.smi_query(vp, rho, gp10, w.srcs, w.recs, stf, kind="rtm")[2]
    nval = 6 * 100 * 100 * 7                        # boundary values a step (faces x cross-section x 2N-1)
    saved = (w.nt - (w.nt - 1) // 10 - 9) * nval * 4
    assert b1 - b10 >= 0.85 * saved            # less the state kept during the continuation


def test_decimation_above_the_rule_is_refused(smi):
    w = S.tiny_2d(nz=45, nx=61, nt=40, nb=10, order=8, src=(12, 30))
    ratio = 5.0 * w.vp.max() / w.vp.min()
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w, dr=int(np.floor(ratio)) + 1), w.srcs,
                        w.recs, _dev(w.stf))
    assert e.value.code == -1
