"""The reverse path (adjoint, source-field reconstruction, imaging and
gradient accumulation) at the benchmark's full grid sizes, against the FP64
oracle, element by element.

The small-grid parity tests cover every mode on grids of 30^3 or less; these
cover the decomposition the full sizes take: the 3D salt RTM grid (300^3 + 20
CPML layers = 340^3, order 8, 150 x 150 receiver carpet) and the 3D
random-medium grid (400 x 400 x 200 + 20 layers, corner source, 200 x 200
carpet), with nt shortened so that the oracle finishes in a minute or two.

- Computing box on: the adjoint box spans the whole receiver carpet (the full
  x-y extent, growing in z), the forward box grows from the source, and the
  reconstruction's box shrinks (Sec. 4.1, Algorithm 2 reverse loop).
- Computing box off: every step covers the whole 340^3 grid, i.e. every tile
  column and y-chunk of the persistent kernels and every piece of the CPML
  bands (the default two-pass kernels), and every interior and CPML-band
  tile of the single-pass step and of the inline-CPML two-pass kernels.

The wavelet is the workload's Ricker advanced so that its main lobe falls
inside the shortened time axis (the workloads delay it by 1.2 / fm, longer
than a 24-step run).  Observed data come from the oracle (a scaled copy of
its seismograms plus seeded noise), never from the GPU.  Bars: images and
gradients 1e-3 relative L2 (FP32 boundaries), the misfit at the bound the
seismogram bar implies.
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


def _early(w, lead):
    """The workload with its Ricker advanced by `lead` samples."""
    w.stf = S.ricker(w.nt + lead, w.dt, w.fm)[lead:].copy()
    return w


def _misfit_ok(J, Jr, seis_ref):
    bound = SEIS_TOL * np.linalg.norm(seis_ref) * np.sqrt(2.0 * Jr) * (1 + SEIS_TOL)
    return abs(J - Jr) <= bound


def _observed(w, **kw):
    ref = O.forward(_oprob(w, **kw), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    rng = np.random.default_rng(11)
    return (0.8 * ref + 0.02 * np.abs(ref).max() * rng.standard_normal(ref.shape)).astype(np.float32)


def test_salt_full_grid_gradient_and_image_box_on(smi):
    """Shot 0 of the salt RTM workload at its full size, 120 steps, box on:
    the FWI gradient, the misfit and the RTM image against the oracle."""
    w = _early(S.salt_3d(nt=120).subset([0]), 60)
    dobs = _observed(w)
    vp, rho, stf, d = _dev(w.vp), _dev(w.rho), _dev(w.stf), _dev(dobs)
    J, g = smi.smi_fwi_gradient(vp, rho, _gprob(smi, w), w.srcs, w.recs, stf, d)
    Jr, gr, ur = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert np.linalg.norm(gr) > 0
    e_g = _rel(g.cpu().numpy(), gr)
    print(f"salt 340^3 box on: gradient {e_g:.2e}, misfit {abs(float(J.item()) - Jr) / Jr:.2e}")
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert e_g <= IMG_TOL
    img = smi.smi_rtm(vp, rho, _gprob(smi, w), w.srcs, w.recs, stf, d)
    _, ir, _ = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs, mode="rtm")
    e_i = _rel(img.cpu().numpy(), ir)
    print(f"salt 340^3 box on: image {e_i:.2e}")
    assert e_i <= IMG_TOL


def test_salt_full_grid_gradient_box_off(smi):
    """Shot 0 of the salt workload, 24 steps with the box off: every tile
    column and y-chunk of the 340^3 grid and every CPML band piece in all
    three modes (forward, adjoint, reconstruction)."""
    w = _early(S.salt_3d(nt=24).subset([0]), 92)
    dobs = _observed(w, use_box=False)
    Jr, gr, ur = O.gradient(_oprob(w, use_box=False), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert np.linalg.norm(gr) > 0
    for kernels in ("auto", "fused", "inline"):   # the three 3D kernel families
        J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w, use_box=False, kernels=kernels),
                                    w.srcs, w.recs, _dev(w.stf), _dev(dobs))
        e_g = _rel(g.cpu().numpy(), gr)
        print(f"salt 340^3 box off ({kernels}): gradient {e_g:.2e}")
        assert _misfit_ok(float(J.item()), Jr, ur)
        assert e_g <= IMG_TOL


def test_random_3d_full_grid_gradient(smi):
    """The 3D random-medium grid (400 x 400 x 200 + 20 layers, corner source,
    40,000 receivers), 100 steps, box on: forward, adjoint over the carpet's
    box, reconstruction and gradient against the oracle."""
    w = _early(S.random_smooth_3d(nt=100), 50)
    dobs = _observed(w)
    J, g = smi.smi_fwi_gradient(_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf),
                                _dev(dobs))
    Jr, gr, ur = O.gradient(_oprob(w), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs)
    assert np.linalg.norm(gr) > 0
    e_g = _rel(g.cpu().numpy(), gr)
    print(f"random 400x400x200: gradient {e_g:.2e}")
    assert _misfit_ok(float(J.item()), Jr, ur)
    assert e_g <= IMG_TOL
