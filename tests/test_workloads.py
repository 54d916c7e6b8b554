"""The seeded synthetic workloads (synth/) against the input recipe they
implement: grid sizes and spacings, time stepping, acquisition counts and
placement, supergather layouts, velocity ranges, the leapfrog stability
margin of the 8th-order stencil, and determinism in the seed.  No arithmetic
of the method is involved."""
import math

import numpy as np
import pytest

import synth

# name: (shape, h, nt, dt, f0, ns, nr, sg_sizes, nsamp, velocity range)
RECIPE = {
    "small2d": ((101, 101), 10.0, 1000, 1e-3, 10.0, 8, 51, [8], 1, (1500.0, 3500.0)),
    "thrust2d": ((187, 801), 25.0, 2000, 2e-3, 8.0, 100, 400, [20] * 5, 16, (2000.0, 6000.0)),
    "salt2d": ((210, 676), 20.0, 2000, 2e-3, 6.0, 130, 676, [26] * 5, 16, (1500.0, 4480.0)),
    "arid2d": ((201, 1001), 10.0, 4000, 5e-4, 15.0, 200, 500, [10, 20, 30, 40, 40, 30, 20, 10], 8, (800.0, 3000.0)),
    "layered3d": ((128, 256, 256), 20.0, 1500, 1.5e-3, 5.0, 64, 4096, [16] * 4, 8, (1500.0, 4500.0)),
}

# largest eigenvalue of the 1D 8th-order second-difference stencil (at kh = pi)
RHO8 = 205 / 72 + 2 * (8 / 5 + 1 / 5 + 8 / 315 + 1 / 560)


@pytest.mark.parametrize("name", sorted(RECIPE))
def test_workload_matches_its_recipe(name):
    shape, h, nt, dt, f0, ns, nr, sg, nsamp, (vmin, vmax) = RECIPE[name]
    w = synth.WORKLOADS[name]()
    assert w.shape == shape and w.hx == w.hz == h and (w.ndim == 2 or w.hy == h)
    assert (w.nt, w.dt, w.f0, w.ns, w.nr, list(w.sg_sizes), w.nsamp) == (nt, dt, f0, ns, nr, sg, nsamp)
    assert (w.vmin, w.vmax) == (vmin, vmax) and w.nb == 20
    assert sum(w.sg_sizes) == w.ns  # the supergathers partition the shots (scale N_s / sum = 1)
    # every source and receiver on a node of the physical grid
    for pts in (w.src, w.rec):
        assert pts.dtype == np.int32 and pts.shape[1] == 3
        assert (pts[:, 0] >= 0).all() and (pts[:, 0] < w.nz).all()
        assert (pts[:, 2] >= 0).all() and (pts[:, 2] < w.nx).all()
        assert (pts[:, 1] >= 0).all() and (pts[:, 1] < max(w.ny, 1)).all()
    assert len({tuple(r) for r in w.rec.tolist()}) == w.nr  # no two receivers on one node
    # leapfrog stability of the 8th-order stencil at the top velocity, with margin
    cfl = vmax * dt * math.sqrt(RHO8 * w.ndim) / h
    assert cfl < 0.9 * 2.0, (name, cfl)


@pytest.mark.parametrize("name", sorted(RECIPE))
def test_models_are_seeded_and_in_range(name):
    w = synth.WORKLOADS[name]()
    m = synth.true_model(w)
    assert m.shape == w.shape and m.dtype == np.float32
    assert m.min() >= w.vmin and m.max() <= w.vmax
    assert m.std() > 0.05 * (w.vmax - w.vmin)  # structure, not a constant
    assert np.array_equal(m, synth.true_model(synth.WORKLOADS[name]()))  # same seed, same model
    other = synth.WORKLOADS[name](seed=w.seed + 1)
    assert not np.array_equal(m, synth.true_model(other))
    s = synth.sample_models(w, 2, seed=5)
    assert s.shape == (2,) + w.shape and s.min() >= w.vmin and s.max() <= w.vmax
    assert np.array_equal(s, synth.sample_models(w, 2, seed=5))


def test_arid_acquisition_follows_the_rough_surface():
    w = synth.arid2d()
    surf = w.extra["surface"]
    m = synth.true_model(w)
    assert (w.src[:, 0] == surf[w.src[:, 2]]).all()                       # sources on the surface
    assert (w.rec[:, 0] == np.minimum(surf[w.rec[:, 2]] + 1, w.nz - 1)).all()  # receivers one cell below
    for ix in range(0, w.nx, 97):  # cells above the surface carry v_min
        assert (m[:surf[ix], ix] == w.vmin).all()


def test_random_records_are_seeded():
    w = synth.small2d(nt=50)
    a, b = synth.random_records(w, 3), synth.random_records(w, 3)
    assert a.shape == (w.ns, w.nt, w.nr) and a.dtype == np.float32 and np.array_equal(a, b)
    assert not np.array_equal(a, synth.random_records(w, 4))


def test_training_patches_are_seeded_normalised_and_shaped():
    import synth.patches as SP
    a = SP.geology_patches(40, 32, 3)
    assert a.shape == (40, 32, 32) and a.dtype == np.float32
    assert a.min() >= -1.0 and a.max() <= 1.0 and np.array_equal(a, SP.geology_patches(40, 32, 3))
    v = SP.volume_patches(20, 16, 4)
    assert v.shape == (20, 16, 16, 16) and v.min() >= -1.0 and v.max() <= 1.0
    assert np.array_equal(v, SP.volume_patches(20, 16, 4)) and not np.array_equal(v, SP.volume_patches(20, 16, 5))


def test_2d_prior_tile_shape_is_tileable_at_every_level():
    from paper_2512_12797_gb300 import unet
    for H, W in [(187, 801), (210, 676), (201, 1001), (64, 64), (101, 101)]:
        Hp, Wp = unet.tile_shape(H, W)
        assert Hp >= H and Wp >= W
        for lev in range(3):
            h, wl = Hp >> lev, Wp >> lev
            assert Hp % (1 << lev) == 0 and Wp % (1 << lev) == 0
            assert wl % 128 == 0 or (wl <= 128 and wl & (wl - 1) == 0)   # the 3x3 kernel's width rule
            assert (h * min(wl, 128)) % 128 == 0                          # whole 128-pixel tiles
    assert unet.tile_shape(187, 801) == (188, 1024)
