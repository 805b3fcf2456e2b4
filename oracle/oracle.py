"""FP64 CPU oracle for staggered-grid acoustic modelling, RTM and FWI gradients.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It wraps
``smi_oracle.c`` (plain C, FP64, written independently of the CUDA library;
the two share no code) through ctypes and builds it with gcc on first use.

Conventions (SMIwiz, arXiv 2311.02293, Secs. 2.1 and 3.4-3.6):
  * model arrays are numpy arrays with z fastest: shape (nx, nz) in 2D and
    (ny, nx, nz) in 3D (the paper's n1 = z, n2 = x, n3 = y);
  * positions are metres (z, x, y) from the first physical node;
  * seismograms are (nt, nrec), sample it holding p^{it+1}.

Functions without an independent pin are marked "parity unpinned" in their
docstring; every other function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "smi_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

ERRORS = {-1: "ORC_ERR_ARG", -2: "ORC_ERR_CFL", -3: "ORC_ERR_DISPERSION", -4: "ORC_ERR_NOMEM"}


class OracleError(RuntimeError):
    def __init__(self, rc: int):
        super().__init__(f"oracle returned {rc} ({ERRORS.get(rc, '?')})")
        self.rc = rc


def build(force: bool = False) -> str:
    """Compile smi_oracle.c into liboracle.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class _Par(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
        ("d1", ctypes.c_double), ("d2", ctypes.c_double), ("d3", ctypes.c_double),
        ("order", ctypes.c_int),
        ("nb", ctypes.c_int),
        ("nt", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("fm", ctypes.c_double),
        ("kaiser_b", ctypes.c_double),
        ("cpml_R", ctypes.c_double),
        ("use_box", ctypes.c_int),
        ("periodic", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("dr", ctypes.c_int),
        ("freesurf", ctypes.c_int),
    ]


@dataclass
class Problem:
    """Grid, time axis and scheme options of one modelling problem."""
    n: tuple            # physical sizes (nz, nx) or (nz, nx, ny)
    d: tuple            # spacings in metres, same order
    nt: int
    dt: float
    order: int = 4
    nb: int = 20
    fm: float = 10.0
    kaiser_b: float = 4.0
    cpml_R: float = 1e-3
    use_box: bool = True
    periodic: bool = False
    nthreads: int = 0
    dr: int = 1         # boundary decimation ratio (Sec. 4.2)
    freesurf: bool = False   # free surface on the top face (image method, Sec. 2.1)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        """numpy shape of a physical model array (slowest axis first)."""
        return tuple(reversed(self.n))

    @property
    def ext_shape(self) -> tuple:
        return tuple(reversed([k + 2 * self.nb for k in self.n]))

    def par(self) -> _Par:
        n = list(self.n) + [1] * (3 - len(self.n))
        d = list(self.d) + [1.0] * (3 - len(self.d))
        return _Par(self.ndim, n[0], n[1], n[2], d[0], d[1], d[2], self.order, self.nb,
                    self.nt, self.dt, self.fm, self.kaiser_b, self.cpml_R, int(self.use_box),
                    int(self.periodic), self.nthreads, self.dr, int(self.freesurf))


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.POINTER(_Par)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        c_int, c_double, c_long = ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.orc_fd_coeffs.argtypes = [c_int, dp]
        L.orc_bessel_i0.argtypes = [c_double]
        L.orc_bessel_i0.restype = c_double
        L.orc_kaiser_1d.argtypes = [c_double, c_int, c_double, ip, dp]
        L.orc_forward.argtypes = [P, dp, dp, dp, dp, c_int, dp, dp, dp]
        L.orc_propagate.argtypes = [P, dp, dp] + [dp] * 10 + [c_int, c_int, dp, dp]
        L.orc_adjoint.argtypes = [P, dp, dp, dp, c_int, dp, dp, c_int, dp]
        L.orc_gradient.argtypes = [P, dp, dp, dp, dp, c_int, dp, dp, c_int, c_int, dp, dp, dp, dp, dp]
        L.orc_reconstruct.argtypes = [P, dp, dp, dp, dp, dp]
        L.orc_check.argtypes = [P, dp, dp]
        L.orc_cpml_profile.argtypes = [P, dp, dp, c_int, c_int, dp, dp]
        L.orc_box_table.argtypes = [P, dp, dp, c_int, dp, c_int, c_int, ip, ip]
        L.orc_band_count.argtypes = [P, dp, dp]
        L.orc_band_count.restype = c_long
        L.orc_max_threads.restype = c_int
        _lib = L
    return _lib


def _d(a):
    """Contiguous float64 copy of a (or None -> NULL)."""
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int):
    if rc != 0:
        raise OracleError(rc)


def _model(prob: Problem, vp, rho):
    vp_a, vp_p = _d(vp)
    rho_a, rho_p = _d(rho)
    size = int(np.prod(prob.n))
    if vp_a.size != size or rho_a.size != size:
        raise ValueError("model arrays do not match the grid")
    return (vp_a, rho_a), vp_p, rho_p


def _pts(pts):
    arr = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
def fd_coeffs(N: int) -> np.ndarray:
    """Staggered FD coefficients a_1..a_N (Sec. 2.1)."""
    a = np.zeros(N)
    _check(lib().orc_fd_coeffs(N, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return a


def bessel_i0(x: float) -> float:
    return lib().orc_bessel_i0(float(x))


def kaiser_1d(x0: float, ri: int, b: float):
    """(first node, weights[2 ri]) of the Kaiser-windowed sinc at x0 (grid units)."""
    first = ctypes.c_int()
    w = np.zeros(2 * ri)
    lib().orc_kaiser_1d(float(x0), ri, float(b), ctypes.byref(first),
                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return first.value, w


def check(prob: Problem, vp, rho) -> int:
    """0, or the negative error the oracle's setup reports (CFL, dispersion, args)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    par = prob.par()
    return lib().orc_check(ctypes.byref(par), vp_p, rho_p)


def cpml_profile(prob: Problem, vp, rho, axis: int, vgrid: bool):
    keep, vp_p, rho_p = _model(prob, vp, rho)
    ne = prob.n[axis] + 2 * prob.nb
    a = np.zeros(ne)
    b = np.zeros(ne)
    par = prob.par()
    _check(lib().orc_cpml_profile(ctypes.byref(par), vp_p, rho_p, axis, int(vgrid),
                                  a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return a, b


def box_table(prob: Problem, vp, rho, pts, n0: int, count: int):
    """Computing-box bounds (extended-grid indices, inclusive) for steps
    n0..n0+count-1 around the stencils of pts: (lo, hi) each [count, 3]
    in axis order z, x, y (Sec. 4.1)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    pa, pp = _pts(pts)
    lo = np.zeros((count, 3), dtype=np.int32)
    hi = np.zeros((count, 3), dtype=np.int32)
    par = prob.par()
    ip = ctypes.POINTER(ctypes.c_int)
    _check(lib().orc_box_table(ctypes.byref(par), vp_p, rho_p, len(pa), pp, n0, count,
                               lo.ctypes.data_as(ip), hi.ctypes.data_as(ip)))
    return lo, hi


def band_count(prob: Problem, vp, rho) -> int:
    keep, vp_p, rho_p = _model(prob, vp, rho)
    par = prob.par()
    n = lib().orc_band_count(ctypes.byref(par), vp_p, rho_p)
    _check(int(n) if n < 0 else 0)
    return int(n)


def forward(prob: Problem, vp, rho, stf, src, rec, snapshots: bool = False):
    """Forward modelling of one shot.  Returns seis (nt, nrec) and, with
    snapshots=True, also p^{it+1} on the physical grid, (nt, *prob.shape)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    stf_a, stf_p = _d(stf)
    assert stf_a.size >= prob.nt
    src_a, src_p = _pts(src)
    rec_a, rec_p = _pts(rec)
    seis = np.zeros((prob.nt, len(rec_a)))
    snap = np.zeros((prob.nt,) + prob.shape) if snapshots else None
    snap_p = snap.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if snapshots else None
    par = prob.par()
    _check(lib().orc_forward(ctypes.byref(par), vp_p, rho_p, stf_p, src_p, len(rec_a), rec_p,
                             seis.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), snap_p))
    return (seis, snap) if snapshots else seis


def propagate(prob: Problem, vp, rho, state: dict, nsteps: int, rec=None):
    """Advance state (dict of extended-size float64 arrays 'p', 'vz', 'vx',
    'vy', optional 'psip_*'/'psiv_*') nsteps steps with no source, over the
    whole grid, in place.  Returns receiver samples (nsteps, nrec) if rec."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    names = ["p", "vz", "vx", "vy", "psip_z", "psip_x", "psip_y", "psiv_z", "psiv_x", "psiv_y"]
    ptrs = []
    for nm in names:
        arr = state.get(nm)
        if arr is None:
            ptrs.append(None)
            continue
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
        ptrs.append(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    nrec = 0
    rec_p = None
    seis = None
    if rec is not None:
        rec_a, rec_p = _pts(rec)
        nrec = len(rec_a)
        seis = np.zeros((nsteps, nrec))
    par = prob.par()
    _check(lib().orc_propagate(ctypes.byref(par), vp_p, rho_p, *ptrs, nsteps, nrec, rec_p,
                               seis.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if seis is not None else None))
    return seis


def adjoint(prob: Problem, vp, rho, src, rec, res, box_mode: int = 0) -> np.ndarray:
    """Adjoint run: returns L^T res as the wavelet-sample vector (nt,)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    src_a, src_p = _pts(src)
    rec_a, rec_p = _pts(rec)
    res_a, res_p = _d(res)
    assert res_a.size == prob.nt * len(rec_a)
    sbar = np.zeros(prob.nt)
    par = prob.par()
    _check(lib().orc_adjoint(ctypes.byref(par), vp_p, rho_p, src_p, len(rec_a), rec_p, res_p,
                             box_mode, sbar.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return sbar


def gradient(prob: Problem, vp, rho, stf, src, rec, dobs, mode: str = "fwi", recon: bool = True,
             with_rho: bool = False, phase_s: np.ndarray | None = None):
    """One shot of Algorithm 2.  mode 'fwi': (misfit, dJ/dVp, seis), and
    with_rho: (misfit, dJ/dVp, seis, dJ/drho at fixed Vp); mode 'rtm':
    (0.0, image, seis); mode 'rtm_norm': (0.0, image normalised by the source
    illumination, seis).  Output arrays have prob.shape.  phase_s (optional,
    float64 array of 4): receives the wall-clock seconds of the forward and
    the reverse time loops after their first steps, then of the two first
    steps (set-up excluded)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    stf_a, stf_p = _d(stf)
    src_a, src_p = _pts(src)
    rec_a, rec_p = _pts(rec)
    dobs_a, dobs_p = _d(dobs)
    assert dobs_a.size == prob.nt * len(rec_a)
    out = np.zeros(prob.shape)
    seis = np.zeros((prob.nt, len(rec_a)))
    g_rho = np.zeros(prob.shape)
    assert not with_rho or mode == "fwi"
    J = ctypes.c_double()
    par = prob.par()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().orc_gradient(ctypes.byref(par), vp_p, rho_p, stf_p, src_p, len(rec_a), rec_p,
                              dobs_p, {"fwi": 0, "rtm": 1, "rtm_norm": 2}[mode], int(recon), ctypes.byref(J),
                              out.ctypes.data_as(dp), seis.ctypes.data_as(dp),
                              g_rho.ctypes.data_as(dp) if with_rho else None,
                              phase_s.ctypes.data_as(dp) if phase_s is not None else None))
    if with_rho:
        return J.value, out, seis, g_rho
    return J.value, out, seis


def reconstruct(prob: Problem, vp, rho, stf, src) -> np.ndarray:
    """Reconstructed source pressure p^{it} on the physical grid, (nt, *shape)."""
    keep, vp_p, rho_p = _model(prob, vp, rho)
    stf_a, stf_p = _d(stf)
    src_a, src_p = _pts(src)
    out = np.zeros((prob.nt,) + prob.shape)
    par = prob.par()
    _check(lib().orc_reconstruct(ctypes.byref(par), vp_p, rho_p, stf_p, src_p,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------------------
# Multi-shot helpers: every shot is independent (Sec. 3.2); images and
# gradients are summed over shots and misfits added (Algorithm 2's final
# reduction).

def forward_shots(prob: Problem, vp, rho, stf, srcs, recs):
    return [forward(prob, vp, rho, stf, s, r) for s, r in zip(srcs, recs)]


def gradient_shots(prob: Problem, vp, rho, stf, srcs, recs, dobs_list, mode="fwi", recon=True):
    total_J = 0.0
    total = np.zeros(prob.shape)
    seis = []
    for s, r, d in zip(srcs, recs, dobs_list):
        J, g, u = gradient(prob, vp, rho, stf, s, r, d, mode=mode, recon=recon)
        total_J += J
        total += g
        seis.append(u)
    return total_J, total, seis
