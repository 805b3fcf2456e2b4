"""Failure detection on the GPU without a fault: the bounded waits of the 3D
tile kernels give up, report SMI_ERR_TIMEOUT, and leave the context usable.

`smi_wait_check` makes one warp wait, with the tile kernels' own wait
helper, on a barrier that nothing completes.  The test runs it with a few
poll limits, checks the status, and then runs a 3D modelling call whose
seismograms must equal those of the same call made before the check.
"""
import numpy as np
import pytest

from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smi():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import smi as mod
    torch.cuda.init()
    return mod


def _forward(smi):
    import torch
    w = S.tiny_3d(nz=28, nx=24, ny=26, nt=40, nb=8, order=8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    return smi.smi_forward(dev(w.vp), dev(w.rho), prob, w.srcs, w.recs, dev(w.stf))[0].cpu().numpy()


def test_bounded_wait_gives_up_and_the_context_stays_usable(smi):
    before = _forward(smi)
    times = {}
    for k in (8, 12, 16):
        rc, ms = smi.smi_wait_check(1 << k)
        assert rc == -6, smi.lib().smi_last_error().decode()
        assert "gave up" in smi.lib().smi_last_error().decode()
        times[k] = ms
    assert times[16] > times[8]
    print("wait check ms by log2(polls):", times, f"~{times[16] / (1 << 16) * 1e6:.1f} ns a poll")
    rc, ms = smi.smi_wait_check(-1)                   # the tile kernels' own limit
    print(f"the tile kernels' limit gives up after {ms:.0f} ms")
    assert rc == -6 and 100.0 < ms < 5000.0           # about a second
    after = _forward(smi)
    assert np.array_equal(before, after)
