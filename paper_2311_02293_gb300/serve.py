"""Serving: continuous batching of modelling / RTM / FWI-gradient requests on
one GPU through the library's request server (include/smi.h, smi_server_*).

``Server`` queues requests of any size, dimension and nt; the library admits
them into worker slots (one CUDA stream each) as slots and device memory
free up, so their work overlaps on the GPU, and merges queued single-shot
requests of one survey into one shot-batched call.  ``make_mix`` draws a
seeded request mix shaped like the serving workload (70 % 2D single-shot
gradient jobs, 30 % 3D forward / RTM shots, orders 4 and 8, FP16
boundaries), as shots of seeded surveys or as independent requests, and
``run_mix`` replays it with Poisson arrivals and reports throughput,
p50/p99 latency and the merges the server made.
"""
from __future__ import annotations

import ctypes
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import smi, synth

_L = smi.lib()


class smi_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("model", smi.smi_model), ("geom", smi.smi_geometry),
                ("wav", smi.smi_wavelet), ("opts", smi.smi_opts), ("dobs", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("misfit", ctypes.c_void_p)]


class smi_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("error", ctypes.c_char * 256)]


_L.smi_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int]
_L.smi_server_create.restype = ctypes.c_void_p
_L.smi_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(smi_request), ctypes.POINTER(ctypes.c_longlong)]
_L.smi_submit.restype = ctypes.c_int
_L.smi_wait.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(smi_result)]
_L.smi_wait.restype = ctypes.c_int
_L.smi_poll.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
_L.smi_poll.restype = ctypes.c_int
_L.smi_cancel.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
_L.smi_cancel.restype = ctypes.c_int
_L.smi_server_info.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_size_t)] * 2 + \
    [ctypes.POINTER(ctypes.c_longlong)] * 3
_L.smi_server_info.restype = ctypes.c_int
_L.smi_server_merges.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_longlong)] * 2
_L.smi_server_merges.restype = ctypes.c_int
_L.smi_server_destroy.argtypes = [ctypes.c_void_p]
_L.smi_server_destroy.restype = None

KINDS = {"forward": 0, "rtm": 1, "gradient": 2}


@dataclass
class Request:
    """One job: a workload (synth.Workload with one shot) and its kind."""
    kind: str
    w: synth.Workload
    prob: smi.Problem
    arrival: float = 0.0          # seconds after the start of the replay
    dobs: object = None           # device tensor (rtm / gradient)
    out: object = None            # device output tensor (set at submission)
    misfit: object = None


class Server:
    def __init__(self, budget_bytes: int = 0, slots: int = 8):
        self._s = _L.smi_server_create(budget_bytes, slots)
        self._keep = {}
        self._lock = threading.Lock()

    def submit(self, kind: str, vp, rho, prob: smi.Problem, srcs, recs, stf, dobs=None, out=None, misfit=None):
        m, keep_m, cuda, shape = smi._model(vp, rho, prob.d)
        geo, keep_g, off = smi._geometry(srcs, recs)
        ks, ps, _ = smi._as_f32(stf)
        w = smi.smi_wavelet(prob.nt, prob.dt, prob.fm, ps)
        o = smi._opts(prob, None)
        r = smi_request()
        r.kind = KINDS[kind]
        r.model, r.geom, r.wav, r.opts = m, geo, w, o
        keep = [keep_m, keep_g, ks, out, misfit]
        if dobs is not None:
            kd, pd, _ = smi._dobs_flat(dobs, cuda, None)
            r.dobs = pd
            keep.append(kd)
        r.out = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        r.misfit = (misfit.data_ptr() if hasattr(misfit, "data_ptr") else misfit.ctypes.data) if misfit is not None else None
        t = ctypes.c_longlong()
        smi._check(_L.smi_submit(self._s, ctypes.byref(r), ctypes.byref(t)))
        with self._lock:
            self._keep[t.value] = (keep, r)
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0) -> dict:
        res = smi_result()
        smi._check(_L.smi_wait(self._s, ticket, timeout, ctypes.byref(res)))
        with self._lock:
            self._keep.pop(ticket, None)
        return {"status": res.status, "device_bytes": res.device_bytes, "t_submit": res.t_submit,
                "t_start": res.t_start, "t_end": res.t_end, "error": res.error.decode()}

    def info(self) -> dict:
        b, u = ctypes.c_size_t(), ctypes.c_size_t()
        q, c, f = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        smi._check(_L.smi_server_info(self._s, ctypes.byref(b), ctypes.byref(u), ctypes.byref(q), ctypes.byref(c),
                                      ctypes.byref(f)))
        mc, mr = ctypes.c_longlong(), ctypes.c_longlong()
        smi._check(_L.smi_server_merges(self._s, ctypes.byref(mc), ctypes.byref(mr)))
        return {"budget": b.value, "in_use": u.value, "queued": q.value, "completed": c.value, "failed": f.value,
                "merged_calls": mc.value, "merged_requests": mr.value}

    def cancel(self, ticket: int) -> bool:
        return _L.smi_cancel(self._s, ticket) == 0

    def close(self):
        if self._s:
            _L.smi_server_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
def _valid(w, prob) -> bool:
    """The library's own set-up checks (CFL, dispersion, geometry)."""
    try:
        smi.smi_query(w.vp, w.rho, prob, w.srcs, w.recs, w.stf, "forward")
        return True
    except smi.SmiError:
        return False


def make_mix(n: int, seed: int = synth.SEED_BASE + 5, scale: float = 1.0, shell: str = "f16",
             surveys: bool = True, n2d: int = 12, n3d: int = 6) -> list:
    """Seeded request mix: 70 % 2D single-shot gradient jobs (nz 201-401,
    nx 601-1601, nt 1500-4000, 12.5 m, 1 ms, 8 Hz), 30 % 3D forward / RTM
    shots (160^3-320^3, nt 1500-3000, 10 m, 0.8 ms, 10 Hz at order 4 or
    12 Hz at order 8), orders 4/8 equally likely.  Grid sizes and nt are
    multiplied by `scale`; draws failing CFL or dispersion are redrawn.

    surveys=True: each request is one shot of a seeded survey -- n2d 2D
    surveys (model, nt, order and 40 shot positions) and n3d 3D surveys
    (model, nt, order and 8 shots) drawn from the ranges above -- so the
    requests of one survey share model, wavelet and options, as the shots of
    an FWI or RTM job do, and the server may run them in one call.
    surveys=False: every request draws its own nt (models from a size-bucket
    cache), so no two requests can share a call."""
    rng = np.random.default_rng(seed)
    if surveys:
        return _survey_mix(n, rng, scale, shell, n2d, n3d)
    cache = {}
    reqs = []
    while len(reqs) < n:
        order = int(rng.choice([4, 8]))
        if rng.random() < 0.7:
            nz = int(rng.integers(201, 402) * scale)
            nx = int(rng.integers(601, 1602) * scale)
            nt = int(rng.integers(1500, 4001) * scale)
            key = ("2d", nz // 20, nx // 50, order)
            if key not in cache:
                cache[key] = synth.layered_fault_2d(nz=nz, nx=nx, nt=nt, nshot=1, order=order,
                                                    seed=synth.SEED_BASE + 50 + len(cache))
            base = cache[key]
            w = synth.Workload(base.name, base.n, base.d, nt, 1e-3, 8.0, order, base.vp, base.rho,
                               base.srcs[:1].copy(), base.recs[:1], vp_true=base.vp_true)
            w.srcs[0, 1] = float(rng.uniform(0.1, 0.9)) * (w.n[1] - 1) * w.d[1]
            w.srcs[0, 1] = round(w.srcs[0, 1] / w.d[1]) * w.d[1]
            kind = "gradient"
        else:
            n3 = int(rng.integers(160, 321) * scale)
            n3 = max(n3 // 20 * 20, 40)
            nt = int(rng.integers(1500, 3001) * scale)
            fm = 10.0 if order == 4 else 12.0
            key = ("3d", n3)
            if key not in cache:
                cache[key] = synth.salt_3d(n=n3, nt=10, nshot=8, seed=synth.SEED_BASE + 60 + len(cache))
            base = cache[key]
            shot = int(rng.integers(0, base.nshot))
            w = synth.Workload(base.name, base.n, base.d, nt, 8e-4, fm, order, base.vp, base.rho,
                               base.srcs[shot:shot + 1], base.recs[shot:shot + 1], vp_true=base.vp_true)
            kind = "forward" if rng.random() < 0.5 else "rtm"
        prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=order, nb=20, shell_prec=shell)
        if not _valid(w, prob):
            continue
        reqs.append(Request(kind, w, prob))
    return reqs


def _survey_mix(n, rng, scale, shell, n2d, n3d) -> list:
    """The survey form of make_mix: surveys first, then requests as shots."""
    s2, s3 = [], []
    while len(s2) < n2d:
        order = int(rng.choice([4, 8]))
        nz = int(rng.integers(201, 402) * scale)
        nx = int(rng.integers(601, 1602) * scale)
        nt = int(rng.integers(1500, 4001) * scale)
        base = synth.layered_fault_2d(nz=nz, nx=nx, nt=nt, nshot=40, order=order,
                                      seed=synth.SEED_BASE + 50 + len(s2))
        h = base.d[1]                     # 40 shots on nodes across 5-95 % of the line
        base.srcs[:, 1] = np.round(np.linspace(0.05, 0.95, 40) * (nx - 1)) * h
        prob = smi.Problem(base.d, nt, 1e-3, 8.0, order=order, nb=20, shell_prec=shell)
        if _valid(base.subset([0]), prob) and _valid(base.subset([39]), prob):
            s2.append((base, order, synth.ricker(nt, 1e-3, 8.0)))
    while len(s3) < n3d:
        order = int(rng.choice([4, 8]))
        n3 = max(int(rng.integers(160, 321) * scale) // 20 * 20, 40)
        nt = int(rng.integers(1500, 3001) * scale)
        fm = 10.0 if order == 4 else 12.0
        base = synth.salt_3d(n=n3, nt=10, nshot=8, seed=synth.SEED_BASE + 60 + len(s3))
        w = synth.Workload(base.name, base.n, base.d, nt, 8e-4, fm, order, base.vp, base.rho, base.srcs[:1],
                           base.recs[:1], vp_true=base.vp_true)
        if _valid(w, smi.Problem(w.d, nt, 8e-4, fm, order=order, nb=20, shell_prec=shell)):
            s3.append((base, order, nt, fm, synth.ricker(nt, 8e-4, fm)))
    reqs = []
    for _ in range(n):
        if rng.random() < 0.7:
            base, order, stf = s2[int(rng.integers(0, n2d))]
            shot = int(rng.integers(0, base.nshot))
            w = synth.Workload(base.name, base.n, base.d, base.nt, 1e-3, 8.0, order, base.vp, base.rho,
                               base.srcs[shot:shot + 1], base.recs[shot:shot + 1], vp_true=base.vp_true, stf=stf)
            kind = "gradient"
        else:
            base, order, nt, fm, stf = s3[int(rng.integers(0, n3d))]
            shot = int(rng.integers(0, base.nshot))
            w = synth.Workload(base.name, base.n, base.d, nt, 8e-4, fm, order, base.vp, base.rho,
                               base.srcs[shot:shot + 1], base.recs[shot:shot + 1], vp_true=base.vp_true, stf=stf)
            kind = "forward" if rng.random() < 0.5 else "rtm"
        reqs.append(Request(kind, w, smi.Problem(w.d, w.nt, w.dt, w.fm, order=order, nb=20, shell_prec=shell)))
    return reqs


def _prepare(reqs, dev):
    """Device inputs and observed data (forward modelling in the true model)."""
    import torch
    models, stfs = {}, {}
    for r in reqs:
        key = id(r.w.vp)
        if key not in models:
            models[key] = (torch.from_numpy(r.w.vp).to(dev), torch.from_numpy(r.w.rho).to(dev),
                           torch.from_numpy(r.w.vp_true if r.w.vp_true is not None else r.w.vp).to(dev))
        r._dev = models[key]
        if id(r.w.stf) not in stfs:       # one device wavelet per survey: its requests may share a call
            stfs[id(r.w.stf)] = torch.from_numpy(r.w.stf).to(dev)
        r._stf = stfs[id(r.w.stf)]
        if r.kind != "forward":
            vp_t = r._dev[2]
            plain = smi.Problem(r.prob.d, r.prob.nt, r.prob.dt, r.prob.fm, order=r.prob.order, nb=r.prob.nb)
            r.dobs = smi.smi_forward(vp_t, r._dev[1], plain, r.w.srcs, r.w.recs, r._stf, flat=True)
    torch.cuda.synchronize()


def _out_for(r, dev):
    import torch
    if r.kind == "forward":
        return torch.empty(r.w.nt * len(r.w.recs[0]), device=dev)
    return torch.empty(int(np.prod(r.w.vp.shape)), device=dev)


def run_alone(reqs, dev) -> tuple:
    """One request at a time (direct calls): (outputs, seconds)."""
    import torch
    outs = []
    t0 = time.perf_counter()
    for r in reqs:
        vp, rho, _ = r._dev
        if r.kind == "forward":
            o = smi.smi_forward(vp, rho, r.prob, r.w.srcs, r.w.recs, r._stf, flat=True)
        elif r.kind == "rtm":
            o = smi.smi_rtm(vp, rho, r.prob, r.w.srcs, r.w.recs, r._stf, r.dobs).reshape(-1)
        else:
            o = smi.smi_fwi_gradient(vp, rho, r.prob, r.w.srcs, r.w.recs, r._stf, r.dobs)[1].reshape(-1)
        outs.append(o)
    torch.cuda.synchronize()
    return outs, time.perf_counter() - t0


def run_mix(reqs, dev, slots: int = 8, budget: int = 0, rate: float | None = None, seed: int = 7) -> dict:
    """Replays reqs through a Server with Poisson arrivals at `rate` requests/s
    (None: all at once).  Returns outputs, latencies and throughput."""
    import torch
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    outs = [_out_for(r, dev) for r in reqs]
    mis = [torch.zeros(1, dtype=torch.float64, device=dev) if r.kind == "gradient" else None for r in reqs]
    torch.cuda.synchronize()
    tickets = [None] * len(reqs)
    with Server(budget, slots) as srv:
        t0 = time.perf_counter()

        def submitter():
            t = 0.0
            for k, r in enumerate(reqs):
                t += gaps[k]
                delay = t0 + t - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                vp, rho, _ = r._dev
                tickets[k] = (srv.submit(r.kind, vp, rho, r.prob, r.w.srcs, r.w.recs, r._stf, dobs=r.dobs,
                                         out=outs[k], misfit=mis[k]), time.perf_counter())

        th = threading.Thread(target=submitter)
        th.start()
        results = []
        for k in range(len(reqs)):
            while tickets[k] is None:
                time.sleep(0.001)
            results.append(srv.wait(tickets[k][0]))
        # latency = the server's own submit-to-end time of each request (waiting
        # on the tickets in order would charge a request for earlier ones)
        lat = [r["t_end"] - r["t_submit"] for r in results]
        th.join()
        elapsed = time.perf_counter() - t0
        info = srv.info()
    torch.cuda.synchronize()
    ok = [r["status"] == 0 for r in results]
    ngrad = sum(1 for r, o in zip(reqs, ok) if o and r.kind == "gradient")
    return {"outputs": outs, "results": results, "latency_s": lat, "seconds": elapsed,
            "requests_per_s": sum(ok) / elapsed, "gradient_shots_per_s": ngrad / elapsed,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "failed": len(reqs) - sum(ok), "merged_calls": info["merged_calls"],
            "merged_requests": info["merged_requests"]}
