"""Thin Python binding of libsmi (include/smi.h): argument marshalling only.

Every step of modelling, imaging and gradient computation runs in the CUDA
library; this module only converts arrays to pointers and structs.  Arrays
may be torch tensors (CUDA or CPU) or numpy arrays.  CUDA inputs give CUDA
outputs; host inputs give numpy outputs, and the library copies between host
and device itself.

Array conventions (SMIwiz, arXiv 2311.02293, Secs. 3.4-3.6): z is the fastest
axis, so a 2D model has shape (nx, nz) and a 3D model (ny, nx, nz); positions
are metres (z, x, y) from the first physical node; each shot's seismogram is
(nt, nrec_s) with sample it holding p at time (it+1) dt.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2311_02293_gb300.build``); importing this module without it
raises ImportError.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is a dependency of the package
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmi.so")

SMI_OK = 0
ERRORS = {
    -1: "SMI_ERR_ARG", -2: "SMI_ERR_CFL", -3: "SMI_ERR_DISPERSION", -4: "SMI_ERR_NOMEM",
    -5: "SMI_ERR_UNSTABLE", -6: "SMI_ERR_TIMEOUT", -7: "SMI_ERR_CUDA", -8: "SMI_ERR_UNSUPPORTED",
}
PREC = {"f32": 0, "fp32": 0, "f16": 1, "fp16": 1, "bf16": 2}


class SmiError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code
        self.message = message


class smi_model(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("n3", ctypes.c_int), ("d1", ctypes.c_double), ("d2", ctypes.c_double),
                ("d3", ctypes.c_double), ("vp", ctypes.c_void_p), ("rho", ctypes.c_void_p)]


class smi_geometry(ctypes.Structure):
    _fields_ = [("nshot", ctypes.c_int), ("src", ctypes.c_void_p),
                ("rec_offset", ctypes.c_void_p), ("rec", ctypes.c_void_p)]


class smi_wavelet(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("dt", ctypes.c_double), ("fm", ctypes.c_double),
                ("stf", ctypes.c_void_p)]


class smi_opts(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("nb", ctypes.c_int), ("freesurf", ctypes.c_int),
                ("dr", ctypes.c_int), ("use_box", ctypes.c_int), ("shell_prec", ctypes.c_int),
                ("kaiser_b", ctypes.c_double), ("cpml_R", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("max_batch", ctypes.c_int),
                ("profile", ctypes.c_int), ("img_norm", ctypes.c_int), ("kernels", ctypes.c_int),
                ("per_shot", ctypes.c_int)]


class smi_stats(ctypes.Structure):
    _fields_ = [("point_updates", ctypes.c_double), ("bytes", ctypes.c_double * 3),
                ("ms", ctypes.c_double * 3), ("steps", ctypes.c_longlong * 3),
                ("kernel_launches", ctypes.c_longlong), ("device_bytes", ctypes.c_double),
                ("band_values", ctypes.c_longlong)]


# C functions exported by libsmi (the names of include/smi.h)
EXPORTS = ["smi_opts_default", "smi_forward", "smi_rtm", "smi_fwi_gradient", "smi_query", "smi_footprint",
           "smi_box_table", "smi_last_stats", "smi_last_error", "smi_version", "smi_forward_noalloc",
           "smi_forward_vjp", "smi_server_create", "smi_submit", "smi_wait", "smi_poll", "smi_cancel",
           "smi_server_info", "smi_server_merges", "smi_server_destroy", "smi_fwi_gradient_family", "smi_wait_check",
           "smi_forward_adjoint", "smi_dot", "smi_forward_tape", "smi_tape_vjp", "smi_tape_free"]
KERNELS = {"auto": 0, "generic": 1, "twopass": 2, "fused": 3, "inline": 4}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    c_int, vp = ctypes.c_int, ctypes.c_void_p
    L.smi_opts_default.argtypes = [P(smi_opts)]
    L.smi_opts_default.restype = None
    common = [P(smi_model), P(smi_geometry), P(smi_wavelet), P(smi_opts)]
    L.smi_forward.argtypes = common + [vp]
    L.smi_forward_noalloc.argtypes = common + [vp]
    L.smi_rtm.argtypes = common + [vp, vp]
    L.smi_fwi_gradient.argtypes = common + [vp, vp, vp]
    L.smi_fwi_gradient_family.argtypes = common + [vp, c_int, c_int, vp, vp, vp]
    L.smi_wait_check.argtypes = [vp, ctypes.c_longlong, P(ctypes.c_double)]
    L.smi_forward_vjp.argtypes = common + [vp, vp]
    L.smi_forward_adjoint.argtypes = common + [vp, vp]
    L.smi_forward_tape.argtypes = common + [vp, P(ctypes.c_void_p)]
    L.smi_tape_vjp.argtypes = [vp, vp, vp, vp]
    L.smi_tape_free.argtypes = [vp]
    L.smi_tape_free.restype = None
    L.smi_dot.argtypes = [vp, vp, ctypes.c_size_t, P(ctypes.c_double), vp]
    L.smi_query.argtypes = common + [c_int, P(ctypes.c_size_t), P(ctypes.c_size_t), P(ctypes.c_size_t)]
    L.smi_footprint.argtypes = common + [c_int, P(ctypes.c_size_t)]
    L.smi_box_table.argtypes = common + [c_int, c_int, c_int, c_int, vp, vp]
    L.smi_last_stats.argtypes = [P(smi_stats)]
    L.smi_last_error.restype = ctypes.c_char_p
    L.smi_version.restype = ctypes.c_char_p
    for name in ("smi_forward", "smi_rtm", "smi_fwi_gradient", "smi_query", "smi_footprint", "smi_box_table",
                 "smi_last_stats", "smi_forward_noalloc", "smi_forward_vjp", "smi_fwi_gradient_family",
                 "smi_wait_check", "smi_forward_adjoint", "smi_dot", "smi_forward_tape", "smi_tape_vjp"):
        getattr(L, name).restype = c_int
    return L


_lib = _load()


def lib():
    return _lib


# ---------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return torch is not None and isinstance(x, torch.Tensor)


def _as_f32(x):
    """(keepalive object, pointer, on_cuda) of a float32 contiguous view of x."""
    if _is_torch(x):
        t = x.detach()
        if t.dtype != torch.float32:
            t = t.float()
        t = t.contiguous()
        return t, t.data_ptr(), t.is_cuda
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    return a, a.ctypes.data, False


def _on_model_device(fn):
    """Run a wrapper with the device of its CUDA model array current, so that
    the stream it passes and the device the library launches on are the ones
    that own the arrays (the library refuses device memory of another
    device)."""
    import contextlib
    import functools

    @functools.wraps(fn)
    def wrapped(vp, *args, **kw):
        ctx = torch.cuda.device(vp.device) if _is_torch(vp) and vp.is_cuda else contextlib.nullcontext()
        with ctx:
            return fn(vp, *args, **kw)
    return wrapped


def _f64_host(x):
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


@dataclass
class Problem:
    """Grid spacing, time axis and scheme options shared by the calls."""
    d: tuple
    nt: int
    dt: float
    fm: float
    order: int = 4
    nb: int = 20
    use_box: bool = True
    shell_prec: str = "f32"
    kaiser_b: float = 4.0
    cpml_R: float = 1e-3
    max_batch: int = 0
    profile: bool = False
    dr: int = 1             # boundary decimation ratio (Sec. 4.2)
    img_norm: bool = False  # smi_rtm: normalise each shot's image by its source illumination
    freesurf: bool = False  # free surface on the top face (image method, Sec. 2.1)
    kernels: str = "auto"   # "generic" / "twopass" / "fused" / "inline": force a kernel family (tests)
    per_shot: bool = False  # smi_rtm / smi_fwi_gradient: each shot's image / gradient / misfit, not the sum


def _geometry(srcs, recs):
    srcs = _f64_host(srcs).reshape(-1, 3)
    nshot = len(srcs)
    if isinstance(recs, (list, tuple)):
        rl = [_f64_host(r).reshape(-1, 3) for r in recs]
    else:
        r = _f64_host(recs).reshape(-1, 3)
        rl = [r] * nshot
    if len(rl) != nshot:
        raise ValueError("one receiver array per shot is required")
    off = np.zeros(nshot + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(r) for r in rl])
    rec = np.ascontiguousarray(np.concatenate(rl, axis=0)) if off[-1] else np.zeros((1, 3))
    geo = smi_geometry(nshot, srcs.ctypes.data, off.ctypes.data, rec.ctypes.data)
    return geo, (srcs, off, rec), off


def _model(vp, rho, d):
    if tuple(vp.shape) != tuple(rho.shape):
        raise ValueError("vp and rho must have the same shape")
    shape = tuple(vp.shape)
    ndim = len(shape)
    if ndim not in (2, 3) or len(d) != ndim:
        raise ValueError("2D (nx, nz) or 3D (ny, nx, nz) model with matching spacings required")
    n = list(reversed(shape)) + [1] * (3 - ndim)
    dd = list(d) + [1.0] * (3 - ndim)
    kv, pv, cv = _as_f32(vp)
    kr, pr, cr = _as_f32(rho)
    m = smi_model(ndim, n[0], n[1], n[2], dd[0], dd[1], dd[2], pv, pr)
    return m, (kv, kr), cv, shape


def _opts(prob: Problem, stream):
    o = smi_opts()
    _lib.smi_opts_default(ctypes.byref(o))
    o.order = prob.order
    o.nb = prob.nb
    o.use_box = int(prob.use_box)
    o.shell_prec = PREC[prob.shell_prec] if isinstance(prob.shell_prec, str) else int(prob.shell_prec)
    o.kaiser_b = prob.kaiser_b
    o.cpml_R = prob.cpml_R
    o.max_batch = prob.max_batch
    o.profile = int(prob.profile)
    o.dr = int(prob.dr)
    o.img_norm = int(prob.img_norm)
    o.freesurf = int(prob.freesurf)
    o.kernels = KERNELS[prob.kernels]
    o.per_shot = int(prob.per_shot)
    if stream is not None:
        o.stream = stream
    elif torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
        o.stream = torch.cuda.current_stream().cuda_stream
    return o


def _check(rc: int):
    if rc != SMI_OK:
        raise SmiError(rc, _lib.smi_last_error().decode())


def _empty(n, like_cuda: bool, dtype=np.float32, device=None):
    if like_cuda:
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        t = torch.empty(n, dtype=tdt, device=device)
        return t, t.data_ptr()
    a = np.empty(n, dtype=dtype)
    return a, a.ctypes.data


def _out(out, n, cuda, device, dtype=np.float32):
    """Caller-provided output (tensor or array, host or device) or a new one."""
    if out is None:
        return _empty(n, cuda, dtype=dtype, device=device)
    if _is_torch(out):
        assert out.is_contiguous() and out.numel() == n
        return out, out.data_ptr()
    assert out.flags.c_contiguous and out.size == n and out.dtype == dtype
    return out, out.ctypes.data


def _split(flat, nt, off):
    return [flat[nt * off[s]: nt * off[s + 1]].reshape(nt, off[s + 1] - off[s]) for s in range(len(off) - 1)]


# ---------------------------------------------------------------------------
@_on_model_device
def smi_forward(vp, rho, prob: Problem, srcs, recs, stf, stream=None, flat=False, out=None):
    """Seismograms of every shot (Sec. 2.1; Algorithm 2 forward loop).
    Returns a list of (nt, nrec_s) arrays (or the flat buffer if flat)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    out, pout = _out(out, int(prob.nt * off[-1]), cuda, vp.device if cuda else None)
    _check(_lib.smi_forward(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), pout))
    return out if flat else _split(out, prob.nt, off)


@_on_model_device
def smi_forward_noalloc(vp, rho, prob: Problem, srcs, recs, stf, out, stream=None, flat=False):
    """smi_forward without device allocations: working memory comes from a
    fixed array inside the library (for callers that may not allocate device
    memory).  vp, rho, stf and the preallocated output `out` must be CUDA
    tensors; calls that overlap on the GPU race on that shared array.  The
    arrays are passed as they are: a tensor that is not CUDA, float32 and
    contiguous is refused (converting it would allocate device memory)."""
    for name, t in (("vp", vp), ("rho", rho), ("stf", stf), ("out", out)):
        if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"smi_forward_noalloc: {name} must be a contiguous float32 CUDA tensor")
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    out, pout = _out(out, int(prob.nt * off[-1]), cuda, vp.device if cuda else None)
    _check(_lib.smi_forward_noalloc(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w),
                                    ctypes.byref(o), pout))
    return out if flat else _split(out, prob.nt, off)


def _dobs_flat(dobs, cuda, device):
    if isinstance(dobs, (list, tuple)):
        if _is_torch(dobs[0]):
            return _as_f32(torch.cat([d.reshape(-1) for d in dobs]))
        return _as_f32(np.concatenate([np.asarray(d, np.float32).reshape(-1) for d in dobs]))
    return _as_f32(dobs.reshape(-1) if hasattr(dobs, "reshape") else dobs)


@_on_model_device
def smi_rtm(vp, rho, prob: Problem, srcs, recs, stf, dobs, stream=None, out=None):
    """Zero-lag cross-correlation image summed over shots (Eq. rtmimage)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    kd, pd, _ = _dobs_flat(dobs, cuda, None)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    ns = len(srcs) if prob.per_shot else 1
    img, pimg = _out(out, ns * int(np.prod(shape)), cuda, vp.device if cuda else None)
    _check(_lib.smi_rtm(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), pd, pimg))
    return img.reshape((ns,) + tuple(shape)) if prob.per_shot else img.reshape(shape)


@_on_model_device
def smi_fwi_gradient(vp, rho, prob: Problem, srcs, recs, stf, dobs, stream=None, out=None):
    """(misfit, dJ/dVp) summed over shots (Eqs. objfwi, gradrhokappa)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    kd, pd, _ = _dobs_flat(dobs, cuda, None)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    ns = len(srcs) if prob.per_shot else 1
    g, pg = _out(out, ns * int(np.prod(shape)), cuda, vp.device if cuda else None)
    J, pJ = _empty(ns, cuda, dtype=np.float64, device=vp.device if cuda else None)
    _check(_lib.smi_fwi_gradient(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w),
                                 ctypes.byref(o), pd, pJ, pg))
    return J, (g.reshape((ns,) + tuple(shape)) if prob.per_shot else g.reshape(shape))


@_on_model_device
def smi_fwi_gradient_family(vp, rho, prob: Problem, srcs, recs, stf, dobs, family: int = 1, log: bool = False,
                            stream=None):
    """(misfit, dJ/dVp, dJ/drho) for family 1, (misfit, dJ/dVp, dJ/dIp) for
    family 2 (Ip = rho Vp); log: gradients with respect to the logarithms."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    kd, pd, _ = _dobs_flat(dobs, cuda, None)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    dev = vp.device if cuda else None
    g1, p1 = _out(None, int(np.prod(shape)), cuda, dev)
    g2, p2 = _out(None, int(np.prod(shape)), cuda, dev)
    J, pJ = _empty(1, cuda, dtype=np.float64, device=dev)
    _check(_lib.smi_fwi_gradient_family(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o),
                                        pd, int(family), int(bool(log)), pJ, p1, p2))
    return J, g1.reshape(shape), g2.reshape(shape)


@_on_model_device
def smi_forward_vjp(vp, rho, prob: Problem, srcs, recs, stf, adj_src, stream=None, out=None):
    """dL/dVp for an upstream gradient adj_src = dL/dseis (seismogram layout)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    kd, pd, _ = _dobs_flat(adj_src, cuda, None)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    g, pg = _out(out, int(np.prod(shape)), cuda, vp.device if cuda else None)
    _check(_lib.smi_forward_vjp(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), pd, pg))
    return g.reshape(shape)


class Tape:
    """The device checkpoint of one smi_forward_tape call (saved boundaries,
    final state, set-up tables), owned by this object; it keeps the model and
    wavelet tensors the call read alive until it is freed."""

    def __init__(self, ptr, keep, shape, device):
        self._p = ptr
        self._keep = keep
        self.shape = shape
        self.device = device

    def vjp(self, adj_src, stream=None, out=None):
        """dL/dVp for dL/dseis = adj_src (seismogram layout); one call per tape."""
        if not self._p:
            raise ValueError("the tape was freed")
        cuda = self.device is not None
        kd, pd, _ = _dobs_flat(adj_src, cuda, None)
        g, pg = _out(out, int(np.prod(self.shape)), cuda, self.device)
        ctx = torch.cuda.device(self.device) if cuda else __import__("contextlib").nullcontext()
        with ctx:
            st = stream if stream is not None else (
                torch.cuda.current_stream().cuda_stream if cuda else None)
            _check(_lib.smi_tape_vjp(self._p, pd, pg, st))
        return g.reshape(self.shape)

    def free(self):
        if self._p:
            _lib.smi_tape_free(self._p)
            self._p = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


@_on_model_device
def smi_forward_tape(vp, rho, prob: Problem, srcs, recs, stf, stream=None):
    """(flat seismograms, Tape): smi_forward that keeps its checkpoint for one
    later reverse pass (Tape.vjp)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    out, pout = _out(None, int(prob.nt * off[-1]), cuda, vp.device if cuda else None)
    t = ctypes.c_void_p()
    _check(_lib.smi_forward_tape(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), pout,
                                 ctypes.byref(t)))
    return out, Tape(t.value, (keep_m, ks), shape, vp.device if cuda else None)


@_on_model_device
def smi_forward_adjoint(vp, rho, prob: Problem, srcs, recs, stf, adj_src, stream=None, out=None):
    """Adjoint of the forward map stf -> seismograms at adj_src (seismogram
    layout): nt samples, summed over shots (the dot-product test's L^T d)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    kd, pd, _ = _dobs_flat(adj_src, cuda, None)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    r, pr = _out(out, int(prob.nt), cuda, vp.device if cuda else None)
    _check(_lib.smi_forward_adjoint(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), pd, pr))
    return r


def smi_dot(a, b, stream=None) -> float:
    """FP64 inner product of two float32 CUDA tensors, reduced on the device."""
    if not (_is_torch(a) and _is_torch(b) and a.is_cuda and b.is_cuda):
        raise ValueError("smi_dot needs CUDA tensors")
    ka, pa, _ = _as_f32(a.reshape(-1))
    kb, pb, _ = _as_f32(b.reshape(-1))
    if ka.numel() != kb.numel():
        raise ValueError("smi_dot: sizes differ")
    out = ctypes.c_double()
    with torch.cuda.device(a.device):
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(_lib.smi_dot(pa, pb, ka.numel(), ctypes.byref(out), st))
    return out.value


def smi_footprint(vp, rho, prob: Problem, srcs, recs, stf, kind: str = "forward") -> int:
    """Device bytes of a call from the sizes alone (no device work, no CFL /
    dispersion / position checks)."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, None)
    c = ctypes.c_size_t()
    k = {"forward": 0, "rtm": 1, "gradient": 2, "vjp": 3, "gradient_family": 4}[kind]
    _check(_lib.smi_footprint(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), k,
                              ctypes.byref(c)))
    return c.value


@_on_model_device
def smi_query(vp, rho, prob: Problem, srcs, recs, stf, kind: str = "forward", stream=None):
    """(seis_elems, image_elems, device_bytes) of a call."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    k = {"forward": 0, "rtm": 1, "gradient": 2, "vjp": 3, "gradient_family": 4}[kind]
    _check(_lib.smi_query(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o), k,
                          ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


@_on_model_device
def smi_box_table(vp, rho, prob: Problem, srcs, recs, stf, shot: int, which: str, n0: int,
                  count: int, stream=None):
    """Device-computed computing-box bounds (lo, hi), each (count, 3) int32."""
    m, keep_m, cuda, shape = _model(vp, rho, prob.d)
    geo, keep_g, off = _geometry(srcs, recs)
    ks, ps, _ = _as_f32(stf)
    w = smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
    o = _opts(prob, stream)
    lo = np.zeros((count, 3), dtype=np.int32)
    hi = np.zeros((count, 3), dtype=np.int32)
    _check(_lib.smi_box_table(ctypes.byref(m), ctypes.byref(geo), ctypes.byref(w), ctypes.byref(o),
                              shot, {"source": 0, "receivers": 1}[which], n0, count,
                              lo.ctypes.data, hi.ctypes.data))
    return lo, hi


def smi_wait_check(polls: int = -1, stream=None):
    """(return code, kernel ms) of the bounded-wait give-up check; the
    expected code is SMI_ERR_TIMEOUT (-6)."""
    ms = ctypes.c_double()
    rc = _lib.smi_wait_check(stream, int(polls), ctypes.byref(ms))
    return rc, ms.value


def smi_last_stats() -> dict:
    st = smi_stats()
    _check(_lib.smi_last_stats(ctypes.byref(st)))
    return {"point_updates": st.point_updates, "bytes": list(st.bytes), "ms": list(st.ms),
            "steps": list(st.steps), "kernel_launches": st.kernel_launches,
            "device_bytes": st.device_bytes, "band_values": st.band_values}


def smi_version() -> str:
    return _lib.smi_version().decode()
