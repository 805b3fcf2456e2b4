"""smi_forward_noalloc: forward modelling for callers that may not allocate
device memory (for example code running where another runtime's caching
allocator already holds the device memory, or a loop that cannot afford an
allocation's synchronisation or failure).  Its working memory is a fixed
array inside the library, so its results must equal smi_forward's on
repeated calls, it must reject problems that do not fit, and a call must
not change the device's free memory.

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4       # the seismogram bar of the parity tests


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


def _cases():
    two = S.layered_fault_2d(nz=60, nx=150, nt=300, nshot=3, order=8)
    two.nb = 12
    two.srcs[:, 1] = [250.0, 900.0, 1600.0]
    three = S.tiny_3d(nz=30, nx=26, ny=22, nt=70, nb=6, off_grid=True)
    return [two, three]


@pytest.mark.parametrize("k", [0, 1])
def test_noalloc_matches_forward_on_two_calls_in_a_row(smi, k):
    import torch
    w = _cases()[k]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    ref = smi.smi_forward(vp, rho, prob, w.srcs, w.recs, stf, flat=True)
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full_like(ref, float("nan"))
        free_before = torch.cuda.mem_get_info()[0]
        smi.smi_forward_noalloc(vp, rho, prob, w.srcs, w.recs, stf, out=out, flat=True)
        torch.cuda.synchronize()
        if call == 1:          # the first call on a device may load the library's array
            assert torch.cuda.mem_get_info()[0] == free_before
        a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= SEIS_TOL * np.linalg.norm(b)


def test_noalloc_rejects_problems_beyond_its_capacity(smi):
    import torch
    n = 2000                                   # ~84 MB of wavefields and model: too large
    vp = torch.full((n, n), 2000.0, device="cuda")
    rho = torch.full((n, n), 1000.0, device="cuda")
    prob = smi.Problem((10.0, 10.0), 10, 1e-3, 10.0)
    out = torch.empty(10, device="cuda")
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward_noalloc(vp, rho, prob, np.array([[100.0, 100.0, 0.0]]),
                                np.array([[100.0, 200.0, 0.0]]), torch.zeros(10, device="cuda"), out=out)
    assert e.value.code == -1 and "at most" in e.value.message


def test_noalloc_rejects_host_arrays(smi):
    """The library itself refuses host pointers (called through the C ABI,
    past the Python wrapper's own check)."""
    import ctypes
    w = _cases()[1]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    m, keep_m, _, _ = smi._model(w.vp, w.rho, prob.d)
    geo, keep_g, off = smi._geometry(w.srcs, w.recs)
    ks, ps, _ = smi._as_f32(w.stf)
    wav = smi.smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = smi._opts(prob, None)
    out = np.zeros(w.nt * int(off[-1]), np.float32)
    rc = smi.lib().smi_forward_noalloc(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(wav), ctypes.byref(o),
                                       out.ctypes.data)
    assert rc == -1 and "device pointers" in smi.lib().smi_last_error().decode()


def test_noalloc_wrapper_refuses_conversions(smi):
    """A float64 or non-contiguous tensor would need a converted copy, which
    allocates device memory: the wrapper refuses it instead."""
    import torch
    w = _cases()[1]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    out = torch.empty(w.nt * len(w.recs[0]), device="cuda")
    with pytest.raises(ValueError):
        smi.smi_forward_noalloc(vp.double(), rho, prob, w.srcs, w.recs, stf, out=out)
    with pytest.raises(ValueError):
        smi.smi_forward_noalloc(vp.transpose(0, 2), rho, prob, w.srcs, w.recs, stf, out=out)


def test_noalloc_free_surface_no_box_unequal_receivers(smi):
    """The host branches of the entry point that the other cases miss: the
    free surface, the computing box off, and shots with different receiver
    counts (per-shot offsets into the output), against smi_forward."""
    import torch
    w = S.tiny_2d(nz=40, nx=50, nt=180, nb=8, order=8, src=(6, 20))
    srcs = np.array([w.srcs[0], w.srcs[0] + np.array([0.0, 120.0, 0.0])])
    recs = [w.recs[0], w.recs[0][::3].copy()]
    assert len(recs[0]) != len(recs[1])
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, use_box=False, freesurf=True)
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    ref = smi.smi_forward(vp, rho, prob, srcs, recs, stf, flat=True)
    out = torch.full_like(ref, float("nan"))
    smi.smi_forward_noalloc(vp, rho, prob, srcs, recs, stf, out=out, flat=True)
    torch.cuda.synchronize()
    a, b = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a))
    assert np.linalg.norm(a - b) <= SEIS_TOL * np.linalg.norm(b)


@pytest.mark.parametrize("k", [0, 1])
def test_noalloc_matches_the_oracle(smi, k):
    """The entry point's seismograms (its own generic kernels) against the
    FP64 oracle directly, shot by shot, at the seismogram bar."""
    import torch
    from oracle import oracle as O
    w = _cases()[k]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    out = torch.empty(w.nt * sum(len(r) for r in w.recs), device="cuda")
    seis = smi.smi_forward_noalloc(_dev(w.vp), _dev(w.rho), prob, w.srcs, w.recs, _dev(w.stf), out=out)
    oprob = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm)
    for s in range(len(w.srcs)):
        ref = O.forward(oprob, w.vp, w.rho, w.stf, w.srcs[s], w.recs[s])
        a = seis[s].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - ref) <= SEIS_TOL * np.linalg.norm(ref)
