"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/fwi.h declares, encodes bit-exactly like the oracle,
and rejects bad grids and geometry before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2512_12797_gb300 import build
    build.build()
    from paper_2512_12797_gb300 import _native
    return _native


def test_library_exports_every_declared_symbol(native):
    L = native.lib()
    for header, exports in [("fwi.h", native.EXPORTS), ("prior.h", native.PRIOR_EXPORTS)]:
        hdr = open(os.path.join(ROOT, "include", header)).read()
        declared = set(re.findall(r"^(?:int|void|const char\*)\s+(\w+)\s*\(", hdr, re.M))
        assert declared, "no declarations parsed in " + header
        assert declared == set(exports), header
        for name in declared:
            assert hasattr(L, name)


def test_encode_bit_exact_with_oracle(native):
    import paper_2512_12797_gb300 as P
    for seed, it, ns in [(0, 0, 1), (1, 2, 8), (12345, 77, 100), (2 ** 63 + 5, 2 ** 40, 130), (9, 3, 576)]:
        pg, wg = P.encode(seed, it, ns)
        po, wo = O.encode(seed, it, ns)
        assert np.array_equal(pg, po) and np.array_equal(wg, wo)


def test_status_strings(native):
    L = native.lib()
    assert L.fwi_status_string(0) == b"ok"
    assert L.fwi_status_string(-2).startswith(b"stability")


def _grid(**over):
    w = synth.small2d()
    d = w.grid_dict()
    d.update(over)
    return native_grid(d), w


def native_grid(d):
    from paper_2512_12797_gb300._native import FwiGrid
    return FwiGrid(**{k: d[k] for k, _ in FwiGrid._fields_})


def _create(native, grid, src, rec):
    src = np.ascontiguousarray(src, np.int32)
    rec = np.ascontiguousarray(rec, np.int32)
    geom = native.FwiGeom(len(src), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(rec),
                          rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    h = ctypes.c_void_p()
    return native.lib().fwi_create(ctypes.byref(grid), ctypes.byref(geom), 4, 1 << 24, ctypes.byref(h))


def test_create_rejects_unstable_time_step(native):
    g, w = _grid(dt=5e-3)          # v dt / h = 1.75 > 0.5546
    assert _create(native, g, w.src, w.rec) == -2


def test_create_rejects_bad_geometry(native):
    g, w = _grid()
    bad = w.rec.copy()
    bad[0, 2] = w.nx                # outside the physical grid
    assert _create(native, g, w.src, bad) == -1
    dup = np.concatenate([w.rec, w.rec[:1]])
    assert _create(native, g, w.src, dup) == -1   # duplicate receiver node
    g2, _ = _grid(ndim=4)
    assert _create(native, g2, w.src, w.rec) == -1


def test_cfl_bound_matches_stencil_spectrum():
    # largest |symbol| of the 1D 8th-order second difference, at k h = pi
    a = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    rho = -(a[0] + 2 * sum(a[k] * np.cos(k * np.pi) for k in range(1, 5)))
    assert abs(rho - 6.501587) < 1e-6
    # isotropic 2D: v dt / h <= sqrt(4 / (2 rho))
    assert abs(np.sqrt(4 / (2 * rho)) - 0.5546) < 1e-4


def test_noalloc_rejects_mis_sized_buffers(native):
    # the binding checks every buffer's size before any device call: the
    # kernels index them from the sizes they are given
    import torch
    import paper_2512_12797_gb300 as P
    d_pred = torch.zeros(2, 3, 10, 4)
    perm, w = P.encode(1, 0, 6)
    with pytest.raises(ValueError, match="d_obs"):
        P.residual_misfit_noalloc(d_pred, torch.zeros(6, 10, 5), perm, w, [2, 2, 2], 1.0)
    with pytest.raises(ValueError, match="supergathers"):
        P.residual_misfit_noalloc(d_pred, torch.zeros(6, 10, 4), perm, w, [3, 3], 1.0)
    with pytest.raises(ValueError, match="misfit"):
        P.residual_misfit_noalloc(d_pred, torch.zeros(6, 10, 4), perm, w, [2, 2, 2], 1.0,
                                  misfit=torch.zeros(3, dtype=torch.float64))
