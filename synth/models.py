"""Seeded synthetic velocity models (m/s) shaped like the paper's benchmark models.

The paper evaluates on SEAM Arid, SEG/EAGE Salt, SEG/EAGE Overthrust (Sec. 3.2)
and BG Compass cubes (Sec. 3.4, Table of acquisition areas).  None of those
models is available here, so each generator below draws a seeded model with the
shape, velocity range and structural style the workload description gives.
Nothing in this module evaluates the wave equation, the misfit or the sampler:
both the CPU oracle and the CUDA path consume these arrays as plain inputs.

Every model is returned as float32 so that the FP64 oracle and the FP32 device
path start from bit-identical velocities.  Arrays are row-major [nz][nx] in 2D
and [nz][ny][nx] in 3D (x contiguous, z the depth axis).
"""
import numpy as np
from scipy.ndimage import gaussian_filter


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def three_layer(nz, nx, seed, v=(1500.0, 2500.0, 3500.0), smooth=2.0):
    """Smooth 3-layer model with seeded sinusoidal interfaces (small 2D case)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None].astype(np.float64)
    x = np.arange(nx)[None, :].astype(np.float64)
    amp = rng.uniform(2.0, 5.0, 2)
    lam = rng.uniform(0.4, 1.0, 2) * nx
    ph = rng.uniform(0, 2 * np.pi, 2)
    z1 = 0.35 * nz + amp[0] * np.sin(2 * np.pi * x / lam[0] + ph[0])
    z2 = 0.70 * nz + amp[1] * np.sin(2 * np.pi * x / lam[1] + ph[1])
    m = np.where(z < z1, v[0], np.where(z < z2, v[1], v[2]))
    if smooth > 0:
        m = gaussian_filter(m, smooth, mode="nearest")
    return _f32(m)


def thrust_belt(nz, nx, seed, vmin=2000.0, vmax=6000.0, nlayers=14, nfaults=3):
    """Folded layers cut by seeded thrust faults (Overthrust-shaped 2D case)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None].astype(np.float64)
    x = np.arange(nx)[None, :].astype(np.float64) + np.zeros((nz, 1))
    fold = (6.0 * np.sin(2 * np.pi * x / rng.uniform(0.3, 0.6) / nx + rng.uniform(0, 6.28))
            + rng.uniform(15, 30) * np.exp(-((x - rng.uniform(0.3, 0.7) * nx) / (0.12 * nx)) ** 2))
    zs = z + fold
    for _ in range(nfaults):
        x0 = rng.uniform(0.15, 0.85) * nx
        dip = rng.uniform(0.5, 1.5)                      # dx per dz of the fault trace
        throw = rng.uniform(6, 14)                       # vertical offset in cells
        hanging = x > x0 + dip * (z - 0.0)
        zs = zs - throw * hanging
    t = np.clip(zs / nz, 0.0, 1.2)
    layer = np.floor(t * nlayers)
    jitter = rng.uniform(-0.5, 0.5, nlayers + 20)
    vl = vmin + (vmax - vmin) * np.clip((layer + jitter[layer.astype(int) + 10]) / nlayers, 0, 1)
    m = gaussian_filter(vl, 0.7, mode="nearest")
    return _f32(np.clip(m, vmin, vmax))


def salt(nz, nx, seed, vtop=1500.0, vbot=4000.0, vsalt=4480.0):
    """Linear-in-depth background plus a seeded star-convex salt body."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None].astype(np.float64)
    x = np.arange(nx)[None, :].astype(np.float64)
    m = vtop + (vbot - vtop) * z / (nz - 1) + 0 * x
    zc, xc = rng.uniform(0.4, 0.55) * nz, rng.uniform(0.35, 0.65) * nx
    r0 = rng.uniform(0.18, 0.25) * nz
    th = np.arctan2((z - zc) * 1.0, (x - xc) / 2.2)
    r = np.hypot(z - zc, (x - xc) / 2.2)
    rb = r0 * (1 + sum(rng.uniform(0.05, 0.18) * np.cos(k * th + rng.uniform(0, 6.28)) for k in range(2, 6)))
    m = np.where(r < rb, vsalt, m)
    return _f32(m)


def arid(nz, nx, seed, vmin=800.0, vmax=3000.0, nvoids=12):
    """Near-surface model: gradient + layers, low-velocity voids, rough topography.

    Cells above a seeded rough surface are set to vmin (no air layer).  Returns
    (model, surface) where surface[ix] is the first subsurface row.
    """
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None].astype(np.float64)
    x = np.arange(nx)[None, :].astype(np.float64)
    base = 1200.0 + (vmax - 1200.0) * (z / (nz - 1)) ** 0.8 + 0 * x
    lay = gaussian_filter(rng.normal(0, 1, (nz, 1)), 2.0) * 250.0
    m = base + lay
    for _ in range(nvoids):
        zc, xc = rng.uniform(0.08, 0.45) * nz, rng.uniform(0, nx)
        a, b = rng.uniform(2, 6), rng.uniform(4, 15)
        m = np.where(((z - zc) / a) ** 2 + ((x - xc) / b) ** 2 < 1.0, rng.uniform(vmin, 1100.0), m)
    surf = 3.0 + gaussian_filter(rng.normal(0, 1, nx), 15.0) * 40.0
    surf = np.clip(np.round(surf - surf.min() + 1), 1, nz // 8).astype(np.int64)
    m = np.where(z < surf[None, :], vmin, m)
    return _f32(np.clip(m, vmin, vmax)), surf


def layered_fault_3d(nz, ny, nx, seed, vmin=1500.0, vmax=4500.0, nlayers=10):
    """Dipping layered volume offset by one seeded planar fault (3D case)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None, None].astype(np.float64)
    y = np.arange(ny)[None, :, None].astype(np.float64)
    x = np.arange(nx)[None, None, :].astype(np.float64)
    dzx, dzy = rng.uniform(-0.08, 0.08, 2)
    zs = z + dzx * (x - nx / 2) + dzy * (y - ny / 2) + 3.0 * np.sin(2 * np.pi * x / (0.7 * nx) + rng.uniform(0, 6.28))
    nrm = rng.normal(0, 1, 3)
    nrm /= np.linalg.norm(nrm)
    side = nrm[0] * (z - nz / 2) + nrm[1] * (y - ny / 2) + nrm[2] * (x - nx / 2) > 0
    zs = zs - rng.uniform(5, 12) * side
    t = np.clip(zs / nz, 0.0, 1.2)
    layer = np.floor(t * nlayers)
    jitter = rng.uniform(-0.4, 0.4, nlayers + 20)
    v = vmin + (vmax - vmin) * np.clip((layer + jitter[layer.astype(int) + 10]) / nlayers, 0, 1)
    return _f32(np.clip(v, vmin, vmax))


def smoothed(model, sigma):
    """Initial model: the true model Gaussian-filtered (Sec. 3.2 initial models)."""
    return _f32(gaussian_filter(model.astype(np.float64), sigma, mode="nearest"))


def homogeneous(shape, v):
    return _f32(np.full(shape, v))


def random_smooth_model(shape, seed, vmin, vmax, sigma=3.0):
    """Smooth random velocity field in [vmin, vmax] (tiny-grid tests)."""
    rng = np.random.default_rng(seed)
    a = gaussian_filter(rng.normal(0, 1, shape), sigma, mode="wrap")
    a = (a - a.min()) / max(a.max() - a.min(), 1e-12)
    return _f32(vmin + (vmax - vmin) * a)
