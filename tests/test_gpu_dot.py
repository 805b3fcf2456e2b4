"""The adjoint dot-product identity on the GPU, in FP64 reductions.

L is the forward map from the wavelet to the seismograms (smi_forward, linear
in the wavelet) and L^T its exact discrete adjoint (smi_forward_adjoint: the
adjoint propagation of Eq. adj with the transposed CPML, sampled with the
source stencil).  For a random wavelet f and random data d,
<L f, d> = <f, L^T d> must hold to FP32 accuracy; both inner products are
reduced on the device in FP64 (smi_dot).  Cases: 2D and 3D, orders 4 and 8,
off-node sources and receivers, the computing box on and off, two shots,
and the free surface.  L^T d is also compared with the oracle's adjoint run
(the same quantity in FP64) at the seismogram bar.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

DOT_TOL = 1e-5
SEIS_TOL = 1e-4


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


CASES = {
    "2d_o4_off": lambda: S.tiny_2d(nz=50, nx=44, nt=150, nb=8, src=(9, 21), off_grid=True),
    "2d_o8_fs": lambda: S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(3, 30), rec_z=1),
    "3d_o4_off": lambda: S.tiny_3d(nz=30, nx=26, ny=22, nt=70, nb=6, off_grid=True),
    "3d_o8": lambda: S.tiny_3d(nz=28, nx=24, ny=26, nt=60, nb=8, order=8),
}


@pytest.mark.parametrize("use_box", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_dot_product_identity_fp64_on_gpu(smi, case, use_box):
    import torch
    w = CASES[case]()
    freesurf = case.endswith("_fs")
    moved = w.srcs.copy()
    moved[:, 1] += 4 * w.d[1]
    srcs = np.concatenate([w.srcs, moved])               # two shots share the wavelet
    recs = [w.recs[0], w.recs[0][::2].copy()]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, use_box=use_box, freesurf=freesurf)
    rng = np.random.default_rng(20231102)
    f = rng.standard_normal(w.nt).astype(np.float32)
    d = rng.standard_normal(w.nt * sum(len(r) for r in recs)).astype(np.float32)
    vp, rho, fd, dd = _dev(w.vp), _dev(w.rho), _dev(f), _dev(d)
    Lf = smi.smi_forward(vp, rho, prob, srcs, recs, fd, flat=True)
    Ltd = smi.smi_forward_adjoint(vp, rho, prob, srcs, recs, fd, dd)
    torch.cuda.synchronize()
    lhs = smi.smi_dot(Lf, dd)
    rhs = smi.smi_dot(fd, Ltd)
    mis = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    print(f"{case} box={use_box}: <Lf,d> = {lhs:.9e}, <f,L^T d> = {rhs:.9e}, mismatch {mis:.2e}")
    assert lhs != 0.0 and mis <= DOT_TOL
    # L^T d against the oracle's adjoint run, shot by shot
    oprob = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm, use_box=use_box,
                      freesurf=freesurf)
    ref = np.zeros(w.nt)
    off = 0
    for s, r in zip(srcs, recs):
        res = d[off: off + w.nt * len(r)].astype(np.float64).reshape(w.nt, len(r))
        ref += O.adjoint(oprob, w.vp, w.rho, s, r, res, box_mode=2 if use_box else 0)
        off += w.nt * len(r)
    got = Ltd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= SEIS_TOL * np.linalg.norm(ref)


def test_dot_reduction_is_fp64(smi):
    """smi_dot keeps FP64 accuracy where an FP32 sum would not: sum of
    1 + k * 2^-30 over 2^22 terms."""
    import torch
    n = 1 << 22
    a = torch.ones(n, device="cuda")
    b = (1.0 + torch.arange(n, device="cuda", dtype=torch.float64) % 8 * 2.0 ** -20).float()
    exact = float(torch.sum(b.double()).item())
    got = smi.smi_dot(a, b)
    assert abs(got - exact) <= 1e-12 * exact
    assert smi.smi_dot(a[:0], b[:0]) == 0.0
