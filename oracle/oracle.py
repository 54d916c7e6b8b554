"""FP64 CPU oracle for the encoded wave-equation likelihood gradient.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  It shares no
code with the CUDA library.  The numerical work happens in fwi_oracle.c
(plain loops, FP64); this module marshals numpy arrays and composes the
steps in the order the paper states them:

  encoded data / operator      sum_{i in B} w_i d_i,  sum_{i in B} w_i F_i(x)     (Sec. 2.1, encoded shots)
  encoded misfit               1/(2 sigma_y^2) ||d~ - F~(x)||^2                   (Sec. 2.1)
  unbiased gradient            (N_s / m) grad Phi~                                (Sec. 2.1)
  Langevin refinement          z - eta grad + nu xi                               (Sec. 2.3 (ii))
  preconditioned refinement    z - eta G d + nu sqrt(G) xi                        (Sec. 2.3 (ii), Sec. 5)
  DDPM re-noise                N(mu~_t(x_t, x0), beta~_t I)                       (Sec. 2.3 (iii))

Readings where the paper is silent are listed in the C file header.  The
supergather scale follows the reading (N_s / sum_j |B_j|) summed over the
supergathers of one sample, which is 1 when the supergathers partition all
shots.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (OpenMP over the spatial loops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
                ("hz", ctypes.c_double), ("hy", ctypes.c_double), ("hx", ctypes.c_double),
                ("nb", ctypes.c_int), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
                ("f0", ctypes.c_double), ("t0", ctypes.c_double),
                ("sponge_vmax", ctypes.c_double), ("sponge_R", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def load(path):
    """ctypes handle with argument types set for every oracle entry point."""
    L = ctypes.CDLL(path)
    G = ctypes.POINTER(_Grid)
    sig = {
        "or_npad": (ctypes.c_long, [G]),
        "or_threads": (ctypes.c_int, [ctypes.c_int]),
        "or_cell_volume": (ctypes.c_double, [G]),
        "or_pad_index": (ctypes.c_long, [G, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "or_sponge": (None, [G, _D]),
        "or_pad_velocity": (None, [G, _D, _D]),
        "or_fold_gradient": (None, [G, _D, _D, _D]),
        "or_lap8": (None, [G, _D, _D]),
        "or_ricker": (None, [G, _D]),
        "or_forward": (ctypes.c_int, [G, _D, ctypes.c_int, _L, _D, ctypes.c_int, _L, _D, _D]),
        "or_adjoint": (ctypes.c_int, [G, _D, _D, ctypes.c_int, _L, _D, ctypes.c_int, _L, _D, _D, _D]),
        "or_tangent": (ctypes.c_int, [G, _D, _D, ctypes.c_int, _L, _D, _D, ctypes.c_int, _L, _D]),
        "or_mix64": (ctypes.c_uint64, [ctypes.c_uint64]),
        "or_splitmix": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
        "or_stream_key": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint64]),
        "or_encode": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int8)]),
        "or_gauss": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]),
        "or_langevin": (None, [_D, _D, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64]),
        "or_langevin_precond": (None, [_D, _D, _D, _D, ctypes.c_int, ctypes.c_long, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_long, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_uint64]),
        "or_renoise": (None, [_D, _D, _D, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_uint64, ctypes.c_uint64]),
        "or_smooth_prior": (ctypes.c_double, [G, _D, _D, ctypes.c_double, ctypes.c_double, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _lp(a):
    return a.ctypes.data_as(_L)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Physical grid + time axis + sponge parameters (one struct for both sides)."""

    def __init__(self, ndim, nz, ny, nx, hz, hy, hx, nb, dt, nt, f0, t0, sponge_vmax, sponge_R=1e-3):
        self.s = _Grid(ndim, nz, ny if ndim == 3 else 1, nx, hz, hy if ndim == 3 else 1.0, hx, nb, dt, nt,
                       f0, t0, sponge_vmax, sponge_R)

    @classmethod
    def from_workload(cls, w, **over):
        d = w.grid_dict()
        d.update(over)
        return cls(**d)

    def __getattr__(self, k):
        return getattr(self.__dict__["s"], k)

    @property
    def ptr(self):
        return ctypes.byref(self.s)

    @property
    def npad(self):
        return lib().or_npad(self.ptr)

    @property
    def pshape(self):
        s = self.s
        if s.ndim == 3:
            return (s.nz + 2 * s.nb, s.ny + 2 * s.nb, s.nx + 2 * s.nb)
        return (s.nz + 2 * s.nb, s.nx + 2 * s.nb)

    @property
    def shape(self):
        s = self.s
        return (s.nz, s.ny, s.nx) if s.ndim == 3 else (s.nz, s.nx)

    @property
    def cell_volume(self):
        return lib().or_cell_volume(self.ptr)

    def with_nt(self, nt):
        s = self.s
        return Grid(s.ndim, s.nz, s.ny, s.nx, s.hz, s.hy, s.hx, s.nb, s.dt, nt, s.f0, s.t0, s.sponge_vmax,
                    s.sponge_R)


# ------------------------------------------------------------------ pieces --

def pad_index(g, pos):
    """Padded linear indices of physical nodes pos[k] = (iz, iy, ix)."""
    pos = np.asarray(pos).reshape(-1, 3)
    return np.array([lib().or_pad_index(g.ptr, int(a), int(b), int(c)) for a, b, c in pos], dtype=np.int64)


def sponge(g):
    out = np.zeros(g.npad)
    lib().or_sponge(g.ptr, _dp(out))
    return out.reshape(g.pshape)


def pad_velocity(g, v):
    v = _f64(v)
    out = np.zeros(g.npad)
    lib().or_pad_velocity(g.ptr, _dp(v), _dp(out))
    return out


def lap8(g, p):
    p = _f64(p).ravel()
    out = np.zeros(g.npad)
    lib().or_lap8(g.ptr, _dp(p), _dp(out))
    return out.reshape(g.pshape)


def ricker(g):
    f = np.zeros(g.nt)
    lib().or_ricker(g.ptr, _dp(f))
    return f


def source_series(g, weights):
    """s_i^n = w_i f(n dt) / cell volume for each weighted source (Sec. 2.1, encoded shots)."""
    f = ricker(g)
    return _f64(np.outer(np.asarray(weights, np.float64), f) / g.cell_volume)


def forward_raw(g, vpad, src_idx, src_ts, rec_idx, keep_snaps=False):
    nr = len(rec_idx)
    d = np.zeros((g.nt, nr))
    snaps = np.zeros((g.nt, g.npad)) if keep_snaps else None
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    src_ts = _f64(src_ts)
    rc = lib().or_forward(g.ptr, _dp(vpad), len(src_idx), _lp(src_idx), _dp(src_ts), nr, _lp(rec_idx),
                          _dp(d), _dp(snaps) if keep_snaps else None)
    if rc != 0:
        raise MemoryError("oracle forward failed (%d)" % rc)
    return (d, snaps) if keep_snaps else d


def adjoint_raw(g, vpad, snaps, src_idx, src_ts, rec_idx, adj, want_grad=True, want_src=False):
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    gc = np.zeros(g.npad) if want_grad else None
    sg = np.zeros((len(src_idx), g.nt)) if want_src else None
    rc = lib().or_adjoint(g.ptr, _dp(vpad), _dp(snaps) if snaps is not None else None, len(src_idx),
                          _lp(src_idx), _dp(_f64(src_ts)), len(rec_idx), _lp(rec_idx), _dp(_f64(adj)),
                          _dp(gc) if want_grad else None, _dp(sg) if want_src else None)
    if rc != 0:
        raise MemoryError("oracle adjoint failed (%d)" % rc)
    return gc, sg


def tangent_raw(g, vpad, snaps, src_idx, src_ts, dc, rec_idx):
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    dd = np.zeros((g.nt, len(rec_idx)))
    rc = lib().or_tangent(g.ptr, _dp(vpad), _dp(snaps), len(src_idx), _lp(src_idx), _dp(_f64(src_ts)),
                          _dp(_f64(dc)), len(rec_idx), _lp(rec_idx), _dp(dd))
    if rc != 0:
        raise MemoryError("oracle tangent failed (%d)" % rc)
    return dd


def fold_gradient(g, v, gc):
    v = _f64(v)
    out = np.zeros(v.size)
    lib().or_fold_gradient(g.ptr, _dp(v), _dp(_f64(gc)), _dp(out))
    return out.reshape(v.shape)


# --------------------------------------------------------------- encoding --

def threads(n=0):
    """Threads of the oracle's spatial loops: n > 0 sets them; returns the
    number in use.  Results do not depend on it (each loop writes disjoint
    elements, and the reductions are serial)."""
    return int(lib().or_threads(int(n)))


def mix64(x):
    return int(lib().or_mix64(ctypes.c_uint64(x & (2 ** 64 - 1))))


def splitmix(s, j):
    return int(lib().or_splitmix(ctypes.c_uint64(s), ctypes.c_uint64(j)))


def encode(seed, it, ns):
    """(perm[ns] int32, w[ns] int8): shot permutation and +-1 weight per shot id."""
    perm = np.zeros(ns, np.int32)
    w = np.zeros(ns, np.int8)
    lib().or_encode(ctypes.c_uint64(seed), ctypes.c_uint64(it), ns,
                    perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return perm, w


def supergathers(perm, sg_sizes):
    """Shot ids of each supergather: consecutive runs of perm."""
    out, o = [], 0
    for s in sg_sizes:
        out.append(np.asarray(perm[o:o + s]))
        o += s
    return out


def gauss(seed, counter, n):
    return np.array([lib().or_gauss(ctypes.c_uint64(seed), ctypes.c_uint64(counter), ctypes.c_uint64(i))
                     for i in range(n)])


# ------------------------------------------------------- composed oracle --

def forward_shot(g, v, src_pos, weights, rec_pos, keep_snaps=False):
    """Record of one (possibly multi-source, weighted) simulation: [nt][nr]."""
    vpad = pad_velocity(g, v)
    return forward_raw(g, vpad, pad_index(g, src_pos), source_series(g, weights), pad_index(g, rec_pos),
                       keep_snaps)


def encoded_forward(g, v, src, rec, perm, w, sg_sizes):
    """F~_j(x) = sum_{i in B_j} w_i F_i(x) as one simulation per supergather: [nsg][nt][nr]."""
    out = []
    for B in supergathers(perm, sg_sizes):
        out.append(forward_shot(g, v, src[B], w[B].astype(np.float64), rec))
    return np.stack(out)


def encoded_data(d_obs, perm, w, sg_sizes):
    """d~_j = sum_{i in B_j} w_i d_i: [nsg][nt][nr]."""
    d_obs = np.asarray(d_obs, np.float64)
    return np.stack([np.tensordot(w[B].astype(np.float64), d_obs[B], axes=1)
                     for B in supergathers(perm, sg_sizes)])


def gradient(g, v, src, rec, d_obs, perm, w, sg_sizes, sigma, scale=None):
    """Encoded misfit and its velocity gradient for one sample.

    Returns (misfit, grad[phys]) with misfit = scale * sum_j Phi~_j and
    grad = scale * sum_j dPhi~_j/dv; scale defaults to N_s / sum_j |B_j|.
    """
    ns = len(src)
    if scale is None:
        scale = ns / float(sum(sg_sizes))
    vpad = pad_velocity(g, v)
    rec_idx = pad_index(g, rec)
    dt_enc = encoded_data(d_obs, perm, w, sg_sizes)
    gc = np.zeros(g.npad)
    phi = 0.0
    for j, B in enumerate(supergathers(perm, sg_sizes)):
        src_idx = pad_index(g, src[B])
        ts = source_series(g, w[B].astype(np.float64))
        d, snaps = forward_raw(g, vpad, src_idx, ts, rec_idx, keep_snaps=True)
        r = d - dt_enc[j]
        phi += 0.5 * float(np.sum(r * r)) / sigma ** 2
        gcj, _ = adjoint_raw(g, vpad, snaps, src_idx, ts, rec_idx, r / sigma ** 2)
        gc += gcj
        del snaps
    return scale * phi, scale * fold_gradient(g, v, gc)


def records_vjp(g, v, src, rec, perm, w, sg_sizes, d_cot):
    """Transposed Jacobian of the encoded records applied to a record
    cotangent, for one sample (the adjoint-state method of Sec. 2.1 with an
    arbitrary adjoint source):  grad[phys] = sum_j (dF~_j/dv)^T d_cot[j].
    """
    vpad = pad_velocity(g, v)
    rec_idx = pad_index(g, rec)
    gc = np.zeros(g.npad)
    for j, B in enumerate(supergathers(perm, sg_sizes)):
        src_idx = pad_index(g, src[B])
        ts = source_series(g, w[B].astype(np.float64))
        _, snaps = forward_raw(g, vpad, src_idx, ts, rec_idx, keep_snaps=True)
        gcj, _ = adjoint_raw(g, vpad, snaps, src_idx, ts, rec_idx, d_cot[j])
        gc += gcj
        del snaps
    return fold_gradient(g, v, gc)


def full_misfit(g, v, src, rec, d_obs, sigma):
    """Full-shot misfit Phi(x) = 1/(2 sigma^2) sum_i ||d_i - F_i(x)||^2 (Sec. 2.1)."""
    phi = 0.0
    for i in range(len(src)):
        d = forward_shot(g, v, src[i:i + 1], [1.0], rec)
        phi += 0.5 * float(np.sum((d - d_obs[i]) ** 2)) / sigma ** 2
    return phi


def langevin(z, grad, eta, nu, vmin, vmax, seed, counter):
    z = _f64(z).copy()
    lib().or_langevin(_dp(z), _dp(_f64(grad)), z.size, eta, nu, vmin, vmax, ctypes.c_uint64(seed),
                      ctypes.c_uint64(counter))
    return z


def langevin_precond(z, grad, v, m, eta, nu, vmin, vmax, seed, counter, k, alpha=0.9, beta1=0.9, eps=1e-3):
    """Preconditioned Langevin step (noise matched to the preconditioner) on
    z [nsamp][...]: returns (z, v, m) updated copies; m None = no first moment."""
    z = _f64(z).copy()
    nsamp = z.shape[0]
    per = z.size // nsamp
    v = _f64(v).copy()
    m = None if m is None else _f64(m).copy()
    lib().or_langevin_precond(_dp(z), _dp(_f64(grad)), _dp(v), _dp(m) if m is not None else None, nsamp, per,
                              alpha, beta1, eps, int(k), eta, nu, vmin, vmax, ctypes.c_uint64(seed),
                              ctypes.c_uint64(counter))
    return z, v, m


def renoise(x_t, x0, abar_t, abar_prev, beta_t, seed, counter):
    x_t = _f64(x_t)
    out = np.zeros_like(x_t)
    lib().or_renoise(_dp(out), _dp(x_t), _dp(_f64(x0)), x_t.size, abar_t, abar_prev, beta_t,
                     ctypes.c_uint64(seed), ctypes.c_uint64(counter))
    return out


def smooth_prior(g, z, zref, lam, mu):
    z = _f64(z)
    grad = np.zeros_like(z)
    phi = lib().or_smooth_prior(g.ptr, _dp(z), _dp(_f64(zref)), lam, mu, _dp(grad))
    return phi, grad


def ddpm_schedule(T=1000, beta1=1e-4, betaT=0.02):
    """Linear beta schedule and cumulative products (Sec. 2.2; T=1000 linear, Sec. 3.1)."""
    beta = np.linspace(beta1, betaT, T)
    abar = np.cumprod(1.0 - beta)
    return beta, abar
