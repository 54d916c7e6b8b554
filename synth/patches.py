"""Seeded training patches for the learned prior (Sec. 2.2: the network is
trained on velocity-model images; Sec. 3.1 trains on patches of geological
models).  The paper's training models are not available; patches are random
crops of the seeded thrust-belt, salt and arid generators of synth.models,
each normalised to [-1, 1] with its generator's velocity range."""
import numpy as np

from . import models

# (generator, model shape (nz, nx), velocity range)
_STYLES = {
    "thrust": (lambda nz, nx, s: models.thrust_belt(nz, nx, s), (187, 801), (2000.0, 6000.0)),
    "salt": (lambda nz, nx, s: models.salt(nz, nx, s), (210, 676), (1500.0, 4480.0)),
    "arid": (lambda nz, nx, s: models.arid(nz, nx, s)[0], (201, 1001), (800.0, 3000.0)),
}


def normalize(v, vmin, vmax):
    return 2.0 * (v - vmin) / (vmax - vmin) - 1.0


def geology_patches(n, size, seed, styles=("thrust", "salt", "arid"), crops_per_model=64):
    """n patches [n, size, size] (float32, normalised units), drawn as random
    crops (with random left-right flips) of seeded models of the given styles."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, size, size), np.float32)
    k = 0
    m = 0
    while k < n:
        style = styles[m % len(styles)]
        gen, (nz, nx), (vmin, vmax) = _STYLES[style]
        model = normalize(gen(nz, nx, int(rng.integers(1 << 30))).astype(np.float64), vmin, vmax)
        for _ in range(min(crops_per_model, n - k)):
            z0 = int(rng.integers(0, nz - size + 1))
            x0 = int(rng.integers(0, nx - size + 1))
            p = model[z0:z0 + size, x0:x0 + size]
            out[k] = p[:, ::-1] if rng.integers(2) else p
            k += 1
        m += 1
    return out


def volume_patches(n, size, seed, model_size=None, crops_per_model=16, vrange=(1500.0, 4500.0)):
    """n volume patches [n, size, size, size] (float32, normalised units) for
    the prior of the 3D models: random crops, with random flips of the two
    horizontal axes, of seeded dipping-layer volumes offset by a planar fault
    (the style of the 3D workload)."""
    rng = np.random.default_rng(seed)
    m = model_size or 2 * size
    out = np.empty((n, size, size, size), np.float32)
    k = 0
    while k < n:
        vol = normalize(models.layered_fault_3d(m, m, m, int(rng.integers(1 << 30)), vrange[0], vrange[1],
                                                nlayers=int(rng.integers(4, 10))).astype(np.float64), *vrange)
        for _ in range(min(crops_per_model, n - k)):
            z0, y0, x0 = (int(rng.integers(0, m - size + 1)) for _ in range(3))
            p = vol[z0:z0 + size, y0:y0 + size, x0:x0 + size]
            if rng.integers(2):
                p = p[:, ::-1, :]
            if rng.integers(2):
                p = p[:, :, ::-1]
            out[k] = p
            k += 1
    return out
