"""Seeded workload descriptions: grids, acquisition geometry, batch shapes.

Each workload fixes a physical grid, time stepping, a Ricker peak frequency,
source/receiver node indices and the supergather layout.  The five named
workloads follow the acquisition descriptions of Sec. 3.2 and the 3D
acquisition table of Sec. 3.4, scaled to the sizes the build targets:

  small2d      101x101 at 10 m, 8 sources, 51 receivers, 10 Hz, dt 1 ms, 1000 steps
  thrust2d     801x187 at 25 m, 100 sources, 400 receivers, 8 Hz, dt 2 ms, 2000 steps,
               16 posterior samples x 5 supergathers of 20 shots
  salt2d       676x210 at 20 m, 130 sources in 5 supergathers of 26, 676 receivers
  arid2d       1001x201 at 10 m, 200 sources, 500 receivers, 15 Hz, dt 0.5 ms, 4000 steps
  layered3d    256x256x128 at 20 m, 64 sources as 4 supergathers of 16, 64x64 receivers

Sources and receivers sit on grid nodes (index = round(depth / h)); the paper
places nodes and sources near the surface at 20-25 m depth.  This module only
lays out inputs; it does no wave-equation arithmetic.
"""
from dataclasses import dataclass, field
import numpy as np

from . import models


@dataclass
class Workload:
    name: str
    ndim: int
    nz: int
    ny: int
    nx: int
    hz: float
    hy: float
    hx: float
    nb: int
    dt: float
    nt: int
    f0: float
    vmin: float
    vmax: float
    src: np.ndarray            # [ns][3] int32 (iz, iy, ix) physical node indices
    rec: np.ndarray            # [nr][3] int32
    sg_sizes: list             # shots per supergather
    nsamp: int                 # posterior samples processed per call
    seed: int = 0
    t0: float = None           # Ricker delay; 1.5 / f0 when None
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        if self.t0 is None:
            self.t0 = 1.5 / self.f0

    @property
    def ns(self):
        return int(self.src.shape[0])

    @property
    def nr(self):
        return int(self.rec.shape[0])

    @property
    def shape(self):
        return (self.nz, self.nx) if self.ndim == 2 else (self.nz, self.ny, self.nx)

    @property
    def padded_points(self):
        p = (self.nz + 2 * self.nb) * (self.nx + 2 * self.nb)
        if self.ndim == 3:
            p *= self.ny + 2 * self.nb
        return p

    def grid_dict(self, sponge_vmax=None):
        """Plain grid description shared by both sides (no derived quantities)."""
        return dict(ndim=self.ndim, nz=self.nz, ny=self.ny if self.ndim == 3 else 1, nx=self.nx,
                    hz=self.hz, hy=self.hy if self.ndim == 3 else 1.0, hx=self.hx, nb=self.nb,
                    dt=self.dt, nt=self.nt, f0=self.f0, t0=self.t0,
                    sponge_vmax=self.vmax if sponge_vmax is None else sponge_vmax, sponge_R=1e-3)


def _line(n, iz, ixs):
    ixs = np.asarray(ixs, dtype=np.int64)
    return np.stack([np.full(len(ixs), iz), np.zeros(len(ixs), np.int64), ixs], 1).astype(np.int32)


def _even(n_items, n_cells, margin=0):
    return np.round(np.linspace(margin, n_cells - 1 - margin, n_items)).astype(np.int64)


def small2d(nt=1000, seed=1000):
    nz = nx = 101
    h = 10.0
    iz = int(round(20.0 / h))
    return Workload("small2d", 2, nz, 1, nx, h, h, h, 20, 1e-3, nt, 10.0, 1500.0, 3500.0,
                    _line(8, iz, _even(8, nx, 5)), _line(51, iz, np.arange(0, nx, 2)),
                    [8], 1, seed)


def thrust2d(nt=2000, seed=2000, nsamp=16):
    nz, nx, h = 187, 801, 25.0
    iz = 1                                        # 25 m
    return Workload("thrust2d", 2, nz, 1, nx, h, h, h, 20, 2e-3, nt, 8.0, 2000.0, 6000.0,
                    _line(100, iz, np.arange(4, nx, 8)[:100]), _line(400, iz, np.arange(0, 800, 2)),
                    [20] * 5, nsamp, seed)


def salt2d(nt=2000, seed=3000, nsamp=16):
    nz, nx, h = 210, 676, 20.0
    iz = 1
    return Workload("salt2d", 2, nz, 1, nx, h, h, h, 20, 2e-3, nt, 6.0, 1500.0, 4480.0,
                    _line(130, iz, _even(130, nx, 2)), _line(676, iz, np.arange(nx)),
                    [26] * 5, nsamp, seed)


def arid2d(nt=4000, seed=4000, nsamp=8, sg_sizes=(10, 20, 30, 40, 40, 30, 20, 10)):
    nz, nx, h = 201, 1001, 10.0
    _, surf = models.arid(nz, nx, seed)
    sx = np.arange(0, nx, 5)[:200]
    rx = np.arange(0, nx, 2)[:500]
    src = np.stack([surf[sx], np.zeros_like(sx), sx], 1).astype(np.int32)
    rec = np.stack([np.minimum(surf[rx] + 1, nz - 1), np.zeros_like(rx), rx], 1).astype(np.int32)
    return Workload("arid2d", 2, nz, 1, nx, h, h, h, 20, 5e-4, nt, 15.0, 800.0, 3000.0,
                    src, rec, list(sg_sizes), nsamp, seed, extra={"surface": surf})


def layered3d(nt=1500, seed=5000, nsamp=8):
    nz, ny, nx, h = 128, 256, 256, 20.0
    iz = 1
    g = np.arange(16, 256, 32)
    sy, sx = np.meshgrid(g, g, indexing="ij")
    src = np.stack([np.full(sx.size, iz), sy.ravel(), sx.ravel()], 1).astype(np.int32)
    r = np.arange(0, 256, 4)
    ry, rx = np.meshgrid(r, r, indexing="ij")
    rec = np.stack([np.full(rx.size, iz), ry.ravel(), rx.ravel()], 1).astype(np.int32)
    return Workload("layered3d", 3, nz, ny, nx, h, h, h, 20, 1.5e-3, nt, 5.0, 1500.0, 4500.0,
                    src, rec, [16] * 4, nsamp, seed)


def tiny2d(nz=31, nx=33, nt=300, ns=4, nr=9, nb=6, h=10.0, dt=1e-3, f0=15.0, nsamp=1, sg_sizes=None, seed=7):
    """Small 2D case for finite-difference and exhaustive checks."""
    iz = 3
    src = _line(ns, iz, _even(ns, nx, 3))
    rec = _line(nr, iz + 2, _even(nr, nx, 1))
    return Workload("tiny2d", 2, nz, 1, nx, h, h, h, nb, dt, nt, f0, 1500.0, 2500.0, src, rec,
                    sg_sizes or [ns], nsamp, seed)


def tiny3d(nz=15, ny=14, nx=13, nt=150, ns=2, nb=4, h=10.0, dt=1e-3, f0=20.0, nsamp=1, seed=9):
    """Small 3D case for finite-difference and adjoint checks."""
    src = np.array([[2, 4, 4], [2, 9, 8]][:ns], dtype=np.int32)
    rec = np.array([[4, y, x] for y in (2, 7, 11) for x in (1, 6, 11)], dtype=np.int32)
    return Workload("tiny3d", 3, nz, ny, nx, h, h, h, nb, dt, nt, f0, 1500.0, 2500.0, src, rec,
                    [ns], nsamp, seed)


WORKLOADS = {"small2d": small2d, "thrust2d": thrust2d, "salt2d": salt2d, "arid2d": arid2d,
             "layered3d": layered3d}


def true_model(w: Workload):
    if w.name == "small2d":
        return models.three_layer(w.nz, w.nx, w.seed)
    if w.name == "thrust2d":
        return models.thrust_belt(w.nz, w.nx, w.seed)
    if w.name == "salt2d":
        return models.salt(w.nz, w.nx, w.seed)
    if w.name == "arid2d":
        return models.arid(w.nz, w.nx, w.seed)[0]
    if w.name == "layered3d":
        return models.layered_fault_3d(w.nz, w.ny, w.nx, w.seed)
    return models.random_smooth_model(w.shape, w.seed, w.vmin, w.vmax)


def initial_model(w: Workload, truth=None):
    truth = true_model(w) if truth is None else truth
    return models.smoothed(truth, 10.0 if w.ndim == 2 else 4.0)


def sample_models(w: Workload, nsamp, seed, spread=0.03):
    """nsamp perturbed copies of the initial model (posterior particles)."""
    base = initial_model(w).astype(np.float64)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsamp):
        pert = models.random_smooth_model(w.shape, int(rng.integers(1 << 31)), -1.0, 1.0, 4.0)
        out.append(np.clip(base * (1 + spread * pert), w.vmin, w.vmax))
    return np.ascontiguousarray(np.stack(out), dtype=np.float32)


def random_records(w: Workload, seed, nshots=None):
    """Seeded band-limited random shot records [ns][nt][nr] (float32).

    Used as observed data where only the arithmetic of the misfit and the
    gradient matters (throughput runs and full-size parity), not the physics.
    """
    ns = w.ns if nshots is None else nshots
    rng = np.random.default_rng(seed)
    from scipy.ndimage import gaussian_filter1d
    d = gaussian_filter1d(rng.normal(0, 1, (ns, w.nt, w.nr)), 3.0, axis=1)
    return np.ascontiguousarray(d * 1e-3, dtype=np.float32)


def add_noise(d, rel, seed):
    """Additive Gaussian noise at `rel` times the data RMS (Sec. 3.2 data generation)."""
    rng = np.random.default_rng(seed)
    rms = float(np.sqrt(np.mean(np.asarray(d, np.float64) ** 2)))
    return np.ascontiguousarray(d + rng.normal(0, rel * rms, d.shape), dtype=np.float32)
