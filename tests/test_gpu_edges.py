"""Edge cases and the full-size workload on the GPU, through the C ABI.

- Degenerate inputs: a shot without receivers, a single time step, and the
  smallest grid the scheme admits (order nodes per axis).  Each is checked
  against the oracle, or against the same call without the degenerate
  shot.
- The 3D random-medium forward workload at full size (400 x 400 x 200,
  corner source, 200 x 200 receivers): every seismogram sample over the
  first 150 steps.
- The 3D salt RTM workload at its full size (300^3 + 20 CPML layers, order
  8, 150 x 150 receiver carpet), in the configuration the bench times:
  - every seismogram sample against the oracle over the first 120 steps
    (the computing box keeps the oracle's work to seconds);
  - the RTM image with the computing box on against off (the box must
    change nothing).
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
    return smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, **kw)


def _oprob(w, **kw):
    return O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm, **kw)


def test_shot_without_receivers(smi):
    """A shot with an empty receiver list records nothing and adds nothing
    to the image or the gradient."""
    w = S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30))
    moved = w.srcs.copy()
    moved[:, 1] += 50.0
    srcs = np.concatenate([w.srcs, moved])
    recs = [w.recs[0], np.zeros((0, 3))]
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    prob = _gprob(smi, w)
    seis = smi.smi_forward(vp, rho, prob, srcs, recs, stf)
    alone = smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf)
    assert seis[1].numel() == 0
    assert np.array_equal(seis[0].cpu().numpy(), alone[0].cpu().numpy())
    dobs = [_dev((0.7 * alone[0].cpu().numpy()).astype(np.float32)), _dev(np.zeros((w.nt, 0), np.float32))]
    img = smi.smi_rtm(vp, rho, prob, srcs, recs, stf, dobs)
    img1 = smi.smi_rtm(vp, rho, prob, w.srcs, w.recs, stf, dobs[0])
    assert np.array_equal(img.cpu().numpy(), img1.cpu().numpy())
    J, g = smi.smi_fwi_gradient(vp, rho, prob, srcs, recs, stf, dobs)
    J1, g1 = smi.smi_fwi_gradient(vp, rho, prob, w.srcs, w.recs, stf, dobs[0])
    assert float(J.item()) == float(J1.item())
    assert np.array_equal(g.cpu().numpy(), g1.cpu().numpy())


@pytest.mark.parametrize("dim", [2, 3])
def test_single_time_step(smi, dim):
    """nt = 1: receivers on and around the (off-grid) source record the one
    injection; the FWI gradient is exactly zero (v^{1/2} = 0, the source
    enters after the pressure update); the RTM image pairs the residual
    with that injection."""
    w = (S.tiny_2d(nz=40, nx=44, nt=1, nb=8, order=8, src=(10, 20), off_grid=True) if dim == 2
         else S.tiny_3d(nz=24, nx=22, ny=20, nt=1, nb=6, order=8, off_grid=True))
    c = w.srcs[0]
    offs = np.array([[0.0, 0.0, 0.0], [w.d[0], 0.0, 0.0], [0.0, -w.d[1], 0.0], [0.5 * w.d[0], 0.5 * w.d[1], 0.0]])
    w.recs = [c + offs]
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))[0]
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(ref) > 0
    assert _rel(seis.cpu().numpy(), ref) <= SEIS_TOL
    dobs = (0.5 * ref).astype(np.float32)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    Jr, gr, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert abs(float(J.item()) - Jr) <= 1e-3 * Jr
    assert np.all(gr == 0.0) and float(g.abs().max()) == 0.0
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    assert _rel(img.cpu().numpy(), ir) <= IMG_TOL


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("dim", [2, 3])
def test_smallest_grid(smi, order, dim):
    """order nodes per axis (the least the stencil admits) and CPML layers
    of order / 2 (the least nb), source in the middle, receivers on every
    node of the second row (2D) or plane (3D, every second node)."""
    n = order
    w = (S.tiny_2d(nz=n, nx=n, nt=40, nb=order // 2, order=order, src=(n // 2, n // 2)) if dim == 2
         else S.tiny_3d(nz=n, nx=n, ny=n, nt=30, nb=order // 2, order=order))
    h = np.array(w.d + (0.0,) * (3 - dim))
    w.srcs = np.array([[(n // 2) * h[0], (n // 2) * h[1], (n // 2) * h[2]]])
    step = 1 if dim == 2 else 2
    w.recs = [np.array([[h[0], ix * h[1], iy * h[2]] for iy in (range(0, n, step) if dim == 3 else [0])
                        for ix in range(0, n, step)])]
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))[0]
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(ref) > 0
    assert _rel(seis.cpu().numpy(), ref) <= SEIS_TOL
    img = smi.smi_rtm(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf),
                      _dev(ref.astype(np.float32)))
    _, iref, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], ref, mode="rtm")
    assert _rel(img.cpu().numpy(), iref) <= IMG_TOL


def test_salt_3d_full_grid_seismograms(smi):
    """The bench's grid and geometry (shot 0 of 8, all 22,500 receivers),
    first 120 steps: every sample against the oracle."""
    w = S.salt_3d(nt=120).subset([0])
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))[0]
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(ref) > 0
    print(f"3D salt 340^3 forward: seismograms {_rel(seis.cpu().numpy(), ref):.2e}")
    assert _rel(seis.cpu().numpy(), ref) <= SEIS_TOL


def test_salt_3d_full_grid_rtm_box_invariance(smi):
    """The bench's RTM (shot 0, 400 steps) with the computing box on and
    off: the box only skips nodes whose values are zero."""
    import torch
    w = S.salt_3d(nt=400).subset([0])
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    dobs = smi.smi_forward(vp, rho, _gprob(smi, w), w.srcs, w.recs, stf)[0].contiguous()
    i_box = smi.smi_rtm(vp, rho, _gprob(smi, w), w.srcs, w.recs, stf, dobs)
    i_all = smi.smi_rtm(vp, rho, _gprob(smi, w, use_box=False), w.srcs, w.recs, stf, dobs)
    err = float(torch.linalg.norm(i_box - i_all) / torch.linalg.norm(i_all))
    print(f"box on vs off: {err:.2e}")
    assert err <= 1e-6


def test_random_3d_full_grid_seismograms(smi):
    """The 3D forward workload's grid and geometry at full size (400 x 400 x
    200 + 20 CPML layers, order 8, corner source, 200 x 200 receivers), first
    150 steps: every sample against the oracle."""
    w = S.random_smooth_3d(nt=150)
    seis = smi.smi_forward(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))[0]
    ref = O.forward(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    assert np.linalg.norm(ref) > 0
    print(f"3D random 400x400x200 forward: seismograms {_rel(seis.cpu().numpy(), ref):.2e}")
    assert _rel(seis.cpu().numpy(), ref) <= SEIS_TOL
