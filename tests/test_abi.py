"""C-ABI checks that need no GPU: the library loads, exports every function
include/smi.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smi.h")


@pytest.fixture(scope="module")
def smi():
    import __graft_entry__
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import smi as mod
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(smi_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("smi_forward", "smi_rtm", "smi_fwi_gradient", "smi_query", "smi_last_error"):
        assert required in names


def test_library_exports_every_declared_function(smi):
    lib = ctypes.CDLL(smi.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(smi.EXPORTS)


def test_version_and_defaults(smi):
    assert "sm_103a" in smi.smi_version()
    o = smi.smi_opts()
    smi.lib().smi_opts_default(ctypes.byref(o))
    assert (o.order, o.nb, o.freesurf, o.dr, o.use_box, o.shell_prec) == (4, 20, 0, 1, 1, 0)
    assert o.kaiser_b == 4.0 and o.cpml_R == 1e-3 and o.max_batch == 0


def _call(smi, **over):
    vp = np.full((30, 30), 2000.0, np.float32)
    rho = np.full((30, 30), 1000.0, np.float32)
    prob = smi.Problem((10.0, 10.0), 10, 1e-3, 10.0)
    for k, v in over.items():
        setattr(prob, k, v)
    return smi.smi_forward(vp, rho, prob, np.array([[50.0, 50.0, 0.0]]),
                           np.array([[50.0, 100.0, 0.0]]), np.zeros(10, np.float32))


@pytest.mark.parametrize("field,value,code", [
    ("order", 6, -1),
    ("nb", 1, -1),
    ("shell_prec", 3, -1),
])
def test_bad_options_rejected_on_host(smi, field, value, code):
    with pytest.raises(smi.SmiError) as e:
        _call(smi, **{field: value})
    assert e.value.code == code


def test_bad_flags_are_refused(smi):
    o = smi.smi_opts()
    smi.lib().smi_opts_default(ctypes.byref(o))
    m = smi.smi_model(2, 30, 30, 1, 10.0, 10.0, 1.0, None, None)
    geo = smi.smi_geometry(0, None, None, None)
    w = smi.smi_wavelet(10, 1e-3, 10.0, None)
    # a free-surface flag other than 0 / 1 and a decimation ratio below 1
    # are argument errors (both refused before any device work)
    for field, value, code in (("freesurf", 2, -1), ("dr", 0, -1)):
        o2 = smi.smi_opts.from_buffer_copy(o)
        setattr(o2, field, value)
        rc = smi.lib().smi_forward(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w),
                                   ctypes.byref(o2), None)
        assert rc == code
        assert smi.lib().smi_last_error().decode()


def test_null_arguments_rejected(smi):
    o = smi.smi_opts()
    smi.lib().smi_opts_default(ctypes.byref(o))
    assert smi.lib().smi_forward(None, None, None, ctypes.byref(o), None) == -1
    m = smi.smi_model(4, 30, 30, 1, 10.0, 10.0, 1.0, None, None)
    geo = smi.smi_geometry(1, None, None, None)
    w = smi.smi_wavelet(10, 1e-3, 10.0, None)
    assert smi.lib().smi_forward(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w),
                                 ctypes.byref(o), None) == -1


def test_family_gradient_arguments_checked_on_host(smi):
    """Family outside {1, 2}, log_param outside {0, 1} and null outputs are
    argument errors, raised before any device work."""
    o = smi.smi_opts()
    smi.lib().smi_opts_default(ctypes.byref(o))
    m = smi.smi_model(2, 30, 30, 1, 10.0, 10.0, 1.0, None, None)
    geo = smi.smi_geometry(0, None, None, None)
    w = smi.smi_wavelet(10, 1e-3, 10.0, None)
    buf = (ctypes.c_float * 900)()
    f = smi.lib().smi_fwi_gradient_family
    args = (ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), None)
    assert f(*args, 0, 0, None, buf, buf) == -1
    assert f(*args, 3, 0, None, buf, buf) == -1
    assert f(*args, 1, 2, None, buf, buf) == -1
    assert f(*args, 2, 0, None, buf, None) == -1
    assert smi.lib().smi_last_error().decode()

