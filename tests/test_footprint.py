"""smi_footprint: the device bytes of a call from the sizes alone, with no
device work (the request server's admission at submission).  CPU tests:
it needs no GPU, it is linear in the number of shots, it orders the call
kinds, and it rejects malformed arguments.  The GPU test checks it against
smi_query, which sizes the call after its device set-up."""
import numpy as np
import pytest

from paper_2311_02293_gb300 import smi, synth


def _fp(w, kind, nshot, **kw):
    p = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, **kw)
    s = w.subset(range(nshot))
    return smi.smi_footprint(w.vp, w.rho, p, s.srcs, s.recs, w.stf, kind)


def test_linear_in_shots_and_ordered_by_kind():
    w = synth.salt_3d(n=60, nt=200, nshot=3)
    f = [_fp(w, "rtm", k) for k in (1, 2, 3)]
    assert f[2] - f[1] == f[1] - f[0] > 0
    assert _fp(w, "forward", 2) < _fp(w, "rtm", 2) == _fp(w, "gradient", 2) < _fp(w, "gradient_family", 2)
    # 16-bit boundary storage halves the saved bands
    assert _fp(w, "rtm", 1, shell_prec="f16") < _fp(w, "rtm", 1)


def test_malformed_arguments_are_refused():
    w = synth.tiny_2d()
    p = smi.Problem(w.d, w.nt, w.dt, w.fm, order=6, nb=w.nb)
    with pytest.raises(smi.SmiError) as e:
        smi.smi_footprint(w.vp, w.rho, p, w.srcs, w.recs, w.stf, "forward")
    assert e.value.code == -1


@pytest.mark.gpu
def test_footprint_matches_query():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    torch.cuda.init()
    for w in (synth.salt_3d(n=60, nt=200, nshot=2), synth.layered_fault_2d(nz=60, nx=150, nt=300, nshot=2)):
        vp, rho, stf = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w.vp, w.rho, w.stf))
        p = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
        for kind in ("forward", "rtm", "gradient"):
            q = smi.smi_query(vp, rho, p, w.srcs, w.recs, stf, kind)[2]
            f = smi.smi_footprint(vp, rho, p, w.srcs, w.recs, stf, kind)
            assert abs(f - q) <= 0.01 * q, (kind, f, q)
