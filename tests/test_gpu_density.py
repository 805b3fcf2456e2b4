"""Gradients of the parametrisation families on the GPU (Sec. 2.2, Eq.
gradrhokappa), through the C ABI, against the FP64 oracle.

- Family 1 (Vp, rho): dJ/dVp equals smi_fwi_gradient's output bit for bit;
  dJ/drho matches the oracle's density gradient (pinned by finite
  differences in tests/test_oracle_density.py) within the gradient bar,
  2D and 3D, orders 4 and 8, box on and off, dr = 1 and dr > 1.
- Family 2 (Vp, Ip) and the log transform: the chain rule applied to the
  oracle's pair.
- Several shots in one batch and one shot per batch agree.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


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
    # name: (workload, options)
    "2d_o4": (lambda: S.tiny_2d(nz=50, nx=44, nt=150, nb=8, src=(9, 21), off_grid=True), {}),
    "2d_o8_nobox": (lambda: S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30)), {"use_box": False}),
    "2d_o8_dr4": (lambda: S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30)), {"dr": 4}),
    "3d_o4": (lambda: S.tiny_3d(nz=26, nx=24, ny=22, nt=50, nb=6, off_grid=True), {}),
    "3d_o8": (lambda: S.tiny_3d(nz=28, nx=24, ny=26, nt=60, nb=8, order=8), {}),
}


def _observed(w, opts):
    """Data from a perturbed density (the residual then carries density
    information)."""
    rng = np.random.default_rng(11)
    rho2 = w.rho.astype(np.float64) * (1.0 + 0.05 * rng.standard_normal(w.rho.shape))
    return O.forward(_oprob(w, **opts), w.vp, rho2, w.stf, w.srcs[0], w.recs[0])


@pytest.fixture(scope="module")
def results(smi):
    out = {}
    for name, (make, opts) in CASES.items():
        w = make()
        dobs = _observed(w, opts)
        Jr, gv, _, gr = O.gradient(_oprob(w, **opts), w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], dobs,
                                   with_rho=True)
        args = (_dev(w.vp), _dev(w.rho), _gprob(smi, w, **opts), w.srcs, w.recs, _dev(w.stf),
                _dev(dobs.astype(np.float32)))
        out[name] = (w, args, Jr, gv, gr)
    return out


@pytest.mark.parametrize("case", sorted(CASES))
def test_family1_matches_oracle(smi, results, case):
    w, args, Jr, gv, gr = results[case]
    J, g1, g2 = smi.smi_fwi_gradient_family(*args, family=1)
    J0, g0 = smi.smi_fwi_gradient(*args)
    assert np.array_equal(g1.cpu().numpy(), g0.cpu().numpy())
    assert float(J.item()) == float(J0.item())
    e1, e2 = _rel(g1.cpu().numpy(), gv), _rel(g2.cpu().numpy(), gr)
    print(f"{case}: dJ/dVp {e1:.2e}  dJ/drho {e2:.2e}")
    assert e1 <= GRAD_TOL and e2 <= GRAD_TOL
    assert abs(float(J.item()) - Jr) <= 1e-3 * Jr


@pytest.mark.parametrize("case", ["2d_o8_nobox", "3d_o4"])
@pytest.mark.parametrize("log", [False, True])
def test_family2_and_log_transform(smi, results, case, log):
    w, args, Jr, gv, gr = results[case]
    vp, rho = w.vp.astype(np.float64), w.rho.astype(np.float64)
    _, g1, g2 = smi.smi_fwi_gradient_family(*args, family=2, log=log)
    ref1 = gv - gr * rho / vp
    ref2 = gr / vp
    if log:
        ref1, ref2 = ref1 * vp, ref2 * rho * vp
    assert _rel(g1.cpu().numpy(), ref1) <= GRAD_TOL
    assert _rel(g2.cpu().numpy(), ref2) <= GRAD_TOL
    _, h1, h2 = smi.smi_fwi_gradient_family(*args, family=1, log=log)
    r1, r2 = (gv * vp, gr * rho) if log else (gv, gr)
    assert _rel(h1.cpu().numpy(), r1) <= GRAD_TOL
    assert _rel(h2.cpu().numpy(), r2) <= GRAD_TOL


def test_batches_agree(smi):
    """Three shots in one batch and one shot per batch (the accumulator is
    shared across batches)."""
    w = S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30))
    srcs = np.concatenate([w.srcs, w.srcs + [[0.0, 60.0, 0.0]], w.srcs + [[40.0, -80.0, 0.0]]])
    recs = [w.recs[0]] * 3
    dobs = [(0.9 * O.forward(_oprob(w), w.vp, w.rho, w.stf, s, recs[0])).astype(np.float32) for s in srcs]
    base = (_dev(w.vp), _dev(w.rho))
    _, a1, a2 = smi.smi_fwi_gradient_family(*base, _gprob(smi, w), srcs, recs, _dev(w.stf), [_dev(d) for d in dobs])
    _, b1, b2 = smi.smi_fwi_gradient_family(*base, _gprob(smi, w, max_batch=1), srcs, recs, _dev(w.stf),
                                            [_dev(d) for d in dobs])
    assert _rel(a2.cpu().numpy(), b2.cpu().numpy().astype(np.float64)) <= 1e-5
    assert _rel(a1.cpu().numpy(), b1.cpu().numpy().astype(np.float64)) <= 1e-5
    ref = sum(O.gradient(_oprob(w), w.vp, w.rho, w.stf, s, recs[0], d.astype(np.float64), with_rho=True)[3]
              for s, d in zip(srcs, dobs))
    assert _rel(a2.cpu().numpy(), ref) <= GRAD_TOL


def test_family_query_counts_the_extra_memory(smi):
    w = S.tiny_2d(nz=45, nx=61, nt=160, nb=10, order=8, src=(12, 30))
    args = (_dev(w.vp), _dev(w.rho), _gprob(smi, w), w.srcs, w.recs, _dev(w.stf))
    b2 = smi.smi_query(*args, kind="gradient")[2]
    b4 = smi.smi_query(*args, kind="gradient_family")[2]
    assert b4 > b2


def test_family_gradient_with_host_buffers(smi, results):
    """Host (numpy) model, wavelet and data in, host gradients out: the same
    numbers as with device buffers."""
    w, args, Jr, gv, gr = results["2d_o8_nobox"]
    J0, a1, a2 = smi.smi_fwi_gradient_family(*args, family=2, log=True)
    host = (w.vp, w.rho, args[2], w.srcs, w.recs, w.stf, args[6].cpu().numpy())
    J1, b1, b2 = smi.smi_fwi_gradient_family(*host, family=2, log=True)
    assert isinstance(b1, np.ndarray) and isinstance(b2, np.ndarray)
    assert np.array_equal(a1.cpu().numpy(), b1) and np.array_equal(a2.cpu().numpy(), b2)
    assert float(J0.item()) == float(J1[0])
