"""The serving mix's host logic (CPU): the survey form draws requests as shots
of a few seeded surveys, so requests of one survey share model arrays,
wavelet and options (the server's condition for sharing a call); the
independent form gives every request its own nt.  The library's validity
check (CFL, dispersion, positions) needs the device, so it is stubbed here;
the GPU tests run the real one."""
import collections

import numpy as np
import pytest

from paper_2311_02293_gb300 import serve


@pytest.fixture
def no_device_check(monkeypatch):
    monkeypatch.setattr(serve, "_valid", lambda w, prob: True)


def _key(r):
    return (id(r.w.vp), id(r.w.stf), r.kind, r.w.nt, r.prob.order, r.prob.shell_prec)


def test_survey_mix_shares_models_and_wavelets(no_device_check):
    reqs = serve.make_mix(256, scale=1.0, surveys=True, n2d=12, n3d=6)
    assert len(reqs) == 256
    kinds = collections.Counter((r.kind, r.w.ndim) for r in reqs)
    assert set(kinds) <= {("gradient", 2), ("forward", 3), ("rtm", 3)}
    assert 0.6 < kinds[("gradient", 2)] / 256 < 0.8          # 70 % 2D gradients
    # every request is one shot; the shots of a survey share its arrays
    assert all(len(r.w.srcs) == 1 for r in reqs)
    groups = collections.Counter(_key(r) for r in reqs)
    assert len({k[0] for k in groups}) <= 12 + 6
    assert max(groups.values()) >= 5                          # calls the server can share
    for r in reqs:
        assert r.w.stf.shape == (r.w.nt,)
        n = r.w.n
        if r.w.ndim == 2:
            assert 201 <= n[0] <= 401 and 601 <= n[1] <= 1601 and 1500 <= r.w.nt <= 4000
            x = r.w.srcs[0, 1]
            assert 0 < x < (n[1] - 1) * r.w.d[1] and abs(x / r.w.d[1] - round(x / r.w.d[1])) < 1e-9
        else:
            assert 160 <= n[0] <= 320 and n[0] == n[1] == n[2] and 1500 <= r.w.nt <= 3000


def test_survey_mix_is_seeded(no_device_check):
    a = serve.make_mix(40, scale=0.25, surveys=True, n2d=3, n3d=2)
    b = serve.make_mix(40, scale=0.25, surveys=True, n2d=3, n3d=2)
    assert [(r.kind, r.w.n, r.w.nt, tuple(r.w.srcs[0])) for r in a] == \
           [(r.kind, r.w.n, r.w.nt, tuple(r.w.srcs[0])) for r in b]
    assert all(np.array_equal(x.w.vp, y.w.vp) for x, y in zip(a, b))


def test_independent_mix_draws_each_requests_own_nt(no_device_check):
    reqs = serve.make_mix(64, scale=1.0, surveys=False)
    groups = collections.Counter(_key(r) for r in reqs)
    assert max(groups.values()) == 1                          # no two requests can share a call
    assert len({r.w.nt for r in reqs}) > 50
