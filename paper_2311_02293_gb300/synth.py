"""Seeded synthetic inputs: velocity/density models, acquisition geometry and
source wavelets shaped like the paper's workloads.

This module is the only code shared by the CUDA path and the CPU oracle: it
holds none of the modelling arithmetic, only input generation.  The paper's
own models (Marmousi, Overthrust; Sec. 5) are not available, so seeded
stand-ins with the same grid shapes, acquisition layouts and velocity ranges
are generated here.  Every generator takes its seed from ``SEED_BASE + k``
for workload k and uses numpy's PCG64.

Array conventions: z is the fastest axis (the paper's n1), so a 2D model has
numpy shape (nx, nz) and a 3D model (ny, nx, nz).  Positions are metres
(z, x, y) from the first physical node.  Seismograms are (nt, nrec).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20231102


def ricker(nt: int, dt: float, fm: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet s(t) = (1 - 2 pi^2 fm^2 tau^2) exp(-pi^2 fm^2 tau^2),
    tau = t - t0, sampled at t = it*dt.  The paper's default source is a Ricker
    wavelet (Sec. 3.5) with no stated delay; t0 = 1.2/fm is used here."""
    if t0 is None:
        t0 = 1.2 / fm
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (np.pi * fm * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


@dataclass
class Workload:
    """One modelling/imaging problem: model, geometry, wavelet, options."""
    name: str
    n: tuple                  # physical sizes (nz, nx[, ny])
    d: tuple                  # spacings (m)
    nt: int
    dt: float
    fm: float
    order: int
    vp: np.ndarray            # float32, shape reversed(n)
    rho: np.ndarray           # float32
    srcs: np.ndarray          # (nshot, 3) metres z, x, y
    recs: list                # per shot (nrec_s, 3) metres
    nb: int = 20
    vp_true: np.ndarray | None = None   # model that generates observed data
    stf: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.stf is None:
            self.stf = ricker(self.nt, self.dt, self.fm)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def nshot(self) -> int:
        return len(self.srcs)

    def subset(self, shots) -> "Workload":
        shots = list(shots)
        return Workload(self.name, self.n, self.d, self.nt, self.dt, self.fm, self.order,
                        self.vp, self.rho, self.srcs[shots], [self.recs[s] for s in shots],
                        self.nb, self.vp_true, self.stf)

    def with_nt(self, nt: int) -> "Workload":
        return Workload(self.name, self.n, self.d, nt, self.dt, self.fm, self.order,
                        self.vp, self.rho, self.srcs, self.recs, self.nb, self.vp_true,
                        self.stf[:nt].copy() if len(self.stf) >= nt else ricker(nt, self.dt, self.fm))


def _grid_points(n, d):
    """Coordinates (metres) of physical node indices along each axis."""
    return [np.arange(k) * h for k, h in zip(n, d)]


def _smooth(a: np.ndarray, sigma_cells) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma_cells, mode="reflect")


# ---------------------------------------------------------------------------
def two_layer_2d(nz=201, nx=201, h=10.0, nt=1000, dt=1e-3, fm=10.0, order=4) -> Workload:
    """2D forward, one shot: 2000 m/s over a 3000 m/s half-space starting at
    z = 1 km (the node at z = 1 km belongs to the lower layer), rho = 1000,
    source at (iz=1, ix=nx//2), receivers at iz=1 on every node."""
    z = np.arange(nz) * h
    col = np.where(z < 1000.0 - 1e-9, 2000.0, 3000.0).astype(np.float32)
    vp = np.broadcast_to(col, (nx, nz)).copy()
    rho = np.full((nx, nz), 1000.0, dtype=np.float32)
    src = np.array([[1 * h, (nx // 2) * h, 0.0]])
    rec = np.stack([np.full(nx, 1 * h), np.arange(nx) * h, np.zeros(nx)], axis=1)
    return Workload("2d_two_layer_201x201", (nz, nx), (h, h), nt, dt, fm, order, vp, rho,
                    src, [rec])


def gardner(vp) -> np.ndarray:
    """Gardner's relation rho = 310 vp^0.25 (kg/m^3, vp in m/s; Gardner et
    al. 1974), the density the paper's multiparameter example uses."""
    return (310.0 * np.asarray(vp, dtype=np.float64) ** 0.25).astype(np.float32)


def layered_fault_2d(nz=301, nx=1001, h=12.5, nt=3000, dt=1e-3, fm=8.0, order=8,
                     nshot=40, seed=SEED_BASE + 2) -> Workload:
    """2D FWI stand-in for Marmousi's shape: 8-15 layers with vp increasing
    from 1500 m/s (clipped to [1500, 4500]), one dipping fault (45-75 deg,
    50-150 m throw of the hanging wall), rho = 1000.  vp_true is the layered
    model; vp is its Gaussian smoothing with sigma = 500 m (the starting
    model).  40 shots at x = 400 + 300 k m, z = 25 m; 1001 receivers at
    z = 25 m on every node."""
    rng = np.random.default_rng(seed)
    nl = min(int(rng.integers(8, 16)), max(2, (nz - 6) // 4))   # small grids hold fewer layers
    # interface depths (cells): sorted uniform with >= 3 cells between them
    while True:
        tops = np.sort(rng.integers(3, nz - 3, size=nl - 1))
        if np.all(np.diff(np.concatenate([[0], tops, [nz]])) >= 3):
            break
    vel = [1500.0]
    for _ in range(nl - 1):
        vel.append(vel[-1] + rng.uniform(50.0, 350.0))
    vel = np.clip(np.array(vel), 1500.0, 4500.0)
    z = np.arange(nz)[None, :].astype(np.float64)            # cells
    x = np.arange(nx)[:, None].astype(np.float64)
    dip = np.deg2rad(rng.uniform(45.0, 75.0))
    xf = rng.uniform(0.25, 0.75) * nx                        # fault trace at the surface
    throw = rng.uniform(50.0, 150.0) / h                     # cells
    # hanging wall: nodes on the side the fault dips towards; its layers
    # are shifted down by the throw
    hanging = x > xf + z / np.tan(dip)
    zz = np.where(hanging, z - throw, z)
    layer = np.searchsorted(tops, zz, side="right")
    vp_true = vel[np.clip(layer, 0, nl - 1)].astype(np.float32)
    vp_true = np.broadcast_to(vp_true, (nx, nz)).copy()
    vp0 = _smooth(vp_true.astype(np.float64), 500.0 / h).astype(np.float32)
    rho = np.full((nx, nz), 1000.0, dtype=np.float32)
    sx = 400.0 + 300.0 * np.arange(nshot)
    srcs = np.stack([np.full(nshot, 2 * h), sx, np.zeros(nshot)], axis=1)
    rec = np.stack([np.full(nx, 2 * h), np.arange(nx) * h, np.zeros(nx)], axis=1)
    return Workload("2d_layered_fault_301x1001", (nz, nx), (h, h), nt, dt, fm, order, vp0, rho,
                    srcs, [rec] * nshot, vp_true=vp_true)


def random_smooth_3d(nz=200, nx=400, ny=400, h=10.0, nt=3000, dt=8e-4, fm=12.0, order=8,
                     seed=SEED_BASE + 3, corr=200.0, vlo=1500.0, vhi=4000.0) -> Workload:
    """3D forward stand-in: a Gaussian random field (white noise smoothed by a
    Gaussian of sigma = corr/sqrt(2), i.e. correlation exp(-r^2/corr^2))
    mapped affinely onto [vlo, vhi]; rho = 1000; one source at the surface
    corner (iz=1, ix=0, iy=0); a receiver carpet on every second node in x
    and y at iz=1."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx, nz))
    f = _smooth(w, corr / np.sqrt(2.0) / h)
    f = (f - f.min()) / (f.max() - f.min())
    vp = (vlo + (vhi - vlo) * f).astype(np.float32)
    rho = np.full(vp.shape, 1000.0, dtype=np.float32)
    srcs = np.array([[1 * h, 0.0, 0.0]])
    ix, iy = np.meshgrid(np.arange(0, nx, 2), np.arange(0, ny, 2), indexing="xy")
    rec = np.stack([np.full(ix.size, 1 * h), ix.ravel() * h, iy.ravel() * h], axis=1)
    return Workload(f"3d_random_{nz}x{nx}x{ny}", (nz, nx, ny), (h, h, h), nt, dt, fm, order,
                    vp, rho, srcs, [rec])


def salt_3d(n=300, h=10.0, nt=2500, dt=8e-4, fm=15.0, order=8, seed=SEED_BASE + 4,
            nshot=8) -> Workload:
    """3D RTM stand-in: a layered 2000-3500 m/s background with a Gaussian
    salt-like body (vp = 4500 where exp(-|x-c|^2 / (2 (400 m)^2)) > 0.5,
    c = (z 1700 m, centre x, centre y)); rho = 1000.  vp_true holds the salt,
    the migration model is the same (migrate in the true model).  8 shots at
    iz=2, (ix, iy) in {75,125,175,225} x {100,200} (for n = 300; scaled with
    n otherwise); a receiver carpet on every second node at iz=2."""
    rng = np.random.default_rng(seed)
    nl = 8
    tops = np.sort(rng.choice(np.arange(5, n - 5), size=nl - 1, replace=False))
    vel = np.linspace(2000.0, 3500.0, nl) + rng.uniform(-60.0, 60.0, nl)
    vel = np.clip(vel, 2000.0, 3500.0)
    z = np.arange(n)
    col = vel[np.searchsorted(tops, z, side="right")]
    vp = np.broadcast_to(col, (n, n, n)).astype(np.float32).copy()
    zc = min(1700.0, 0.57 * (n - 1) * h)
    c = np.array([zc, 0.5 * (n - 1) * h, 0.5 * (n - 1) * h])
    zz = (np.arange(n) * h - c[0])[None, None, :]
    xx = (np.arange(n) * h - c[1])[None, :, None]
    yy = (np.arange(n) * h - c[2])[:, None, None]
    r2 = zz * zz + xx * xx + yy * yy
    vp[np.exp(-r2 / (2.0 * 400.0 ** 2)) > 0.5] = 4500.0
    rho = np.full(vp.shape, 1000.0, dtype=np.float32)
    sc = n / 300.0
    pts = [(ix, iy) for iy in (100, 200) for ix in (75, 125, 175, 225)][:nshot]
    srcs = np.array([[2 * h, round(ix * sc) * h, round(iy * sc) * h] for ix, iy in pts])
    ix, iy = np.meshgrid(np.arange(0, n, 2), np.arange(0, n, 2), indexing="xy")
    rec = np.stack([np.full(ix.size, 2 * h), ix.ravel() * h, iy.ravel() * h], axis=1)
    return Workload(f"3d_salt_{n}^3", (n, n, n), (h, h, h), nt, dt, fm, order, vp, rho,
                    srcs, [rec] * len(srcs), vp_true=vp)


def tiny_2d(nz=24, nx=20, h=10.0, nt=60, dt=1e-3, fm=12.0, order=4, nb=6, seed=SEED_BASE + 10,
            src=(5, 9), rec_z=4, rec_step=2, off_grid=False) -> Workload:
    """Small random 2D model for oracle self-tests and GPU parity (a smooth
    random vp in [1800, 2600] and a random rho in [1500, 2500])."""
    rng = np.random.default_rng(seed)
    vp = (1800.0 + 800.0 * rng.random((nx, nz)))
    vp = _smooth(vp, 1.5)
    vp = (1800.0 + 800.0 * (vp - vp.min()) / max(vp.max() - vp.min(), 1e-9)).astype(np.float32)
    rho = (1500.0 + 1000.0 * rng.random((nx, nz))).astype(np.float32)
    dz = 0.37 * h if off_grid else 0.0
    srcs = np.array([[src[0] * h + dz, src[1] * h + 0.61 * dz, 0.0]])
    rx = np.arange(1, nx - 1, rec_step)
    rec = np.stack([np.full(rx.size, rec_z * h + 0.5 * dz), rx * h, np.zeros(rx.size)], axis=1)
    return Workload("2d_tiny", (nz, nx), (h, h), nt, dt, fm, order, vp, rho, srcs, [rec], nb=nb)


def tiny_3d(nz=14, nx=12, ny=10, h=10.0, nt=40, dt=1e-3, fm=12.0, order=4, nb=5,
            seed=SEED_BASE + 11, off_grid=False) -> Workload:
    """Small random 3D model for oracle self-tests and GPU parity."""
    rng = np.random.default_rng(seed)
    vp = (1800.0 + 800.0 * rng.random((ny, nx, nz)))
    vp = _smooth(vp, 1.0)
    vp = (1800.0 + 800.0 * (vp - vp.min()) / max(vp.max() - vp.min(), 1e-9)).astype(np.float32)
    rho = (1500.0 + 1000.0 * rng.random((ny, nx, nz))).astype(np.float32)
    dz = 0.29 * h if off_grid else 0.0
    srcs = np.array([[4 * h + dz, 5 * h + 0.5 * dz, 4 * h + 0.7 * dz]])
    ix, iy = np.meshgrid(np.arange(1, nx - 1, 3), np.arange(1, ny - 1, 3), indexing="xy")
    rec = np.stack([np.full(ix.size, 3 * h + dz), ix.ravel() * h, iy.ravel() * h], axis=1)
    return Workload("3d_tiny", (nz, nx, ny), (h, h, h), nt, dt, fm, order, vp, rho, srcs, [rec],
                    nb=nb)


WORKLOADS = {
    "2d_two_layer": two_layer_2d,
    "2d_layered_fault": layered_fault_2d,
    "3d_random": random_smooth_3d,
    "3d_salt": salt_3d,
}
