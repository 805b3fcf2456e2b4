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
    w = _cases()[1]
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    out = np.zeros(w.nt * len(w.recs[0]), np.float32)
    with pytest.raises(smi.SmiError) as e:
        smi.smi_forward_noalloc(w.vp, w.rho, prob, w.srcs, w.recs, w.stf, out=out)
    assert e.value.code == -1 and "device pointers" in e.value.message
