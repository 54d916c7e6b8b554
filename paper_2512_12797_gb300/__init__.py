"""GB300-native encoded wave-equation likelihood gradient for diffusion-based
posterior sampling in FWI (arXiv 2512.12797).

Thin Python binding over the C ABI of libfwi.so (include/fwi.h).  This module
only marshals arguments: every step of the forward, residual, adjoint and
imaging computation runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.
"""
import ctypes

import numpy as np

from ._native import FwiError, FwiGeom, FwiGrid, check, lib, LIB_PATH, EXPORTS  # noqa: F401

__all__ = ["FWI", "encode", "langevin_step", "renoise", "residual_misfit_noalloc", "FwiError", "EXPORTS"]


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _numel(t, n, name):
    """Every device buffer's size is checked here: the kernels trust it."""
    if t.numel() != n:
        raise ValueError("%s has %d elements (shape %s), expected %d" % (name, t.numel(), tuple(t.shape), n))


def encode(seed, it, ns):
    """Supergather encoding of FWI iteration `it`: (perm int32[ns], w int8[ns]) (fwi_encode)."""
    perm = np.zeros(ns, np.int32)
    w = np.zeros(ns, np.int8)
    check(lib().fwi_encode(ctypes.c_uint64(seed), ctypes.c_uint64(it), int(ns),
                           perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))), "fwi_encode")
    return perm, w


class FWI:
    """One grid + acquisition geometry with its device workspace (fwi_create).

    grid: dict with ndim, nz, ny, nx, hz, hy, hx, nb, dt, nt, f0, t0,
    sponge_vmax, sponge_R.  src/rec: int arrays [n][3] of (iz, iy, ix) nodes.
    """

    def __init__(self, grid, src, rec, max_wavefields, budget_bytes=0):
        self.grid = dict(grid)
        g = FwiGrid(**{k: self.grid[k] for k, _ in FwiGrid._fields_})
        self._src = np.ascontiguousarray(src, np.int32).reshape(-1, 3)
        self._rec = np.ascontiguousarray(rec, np.int32).reshape(-1, 3)
        geom = FwiGeom(len(self._src), self._src.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       len(self._rec), self._rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        h = ctypes.c_void_p()
        check(lib().fwi_create(ctypes.byref(g), ctypes.byref(geom), int(max_wavefields), int(budget_bytes),
                               ctypes.byref(h)), "fwi_create")
        self._h = h
        self.ns, self.nr, self.nt = len(self._src), len(self._rec), int(grid["nt"])
        self.shape = (grid["nz"], grid["nx"]) if grid["ndim"] == 2 else (grid["nz"], grid["ny"], grid["nx"])
        self.phys = int(np.prod(self.shape))

    def close(self):
        """Frees the context's device workspace (also on garbage collection)."""
        if getattr(self, "_h", None):
            lib().fwi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _enc(self, nsamp, perm, w, sg_sizes):
        perm = np.ascontiguousarray(np.broadcast_to(np.asarray(perm, np.int32), (nsamp, self.ns)))
        w = np.ascontiguousarray(np.broadcast_to(np.asarray(w, np.int8), (nsamp, self.ns)))
        sg = np.ascontiguousarray(sg_sizes, np.int32)
        return (perm, w, sg, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), sg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))

    def forward(self, vel, perm, w, sg_sizes, out=None, stream=None):
        """Encoded records F~_j(x): [nsamp][nsg][nt][nr] float32 (fwi_forward)."""
        torch = _torch()
        nsamp = vel.shape[0]
        keep = self._enc(nsamp, perm, w, sg_sizes)
        nsg = len(keep[2])
        _numel(vel, nsamp * self.phys, "vel")
        if out is None:
            out = torch.empty((nsamp, nsg, self.nt, self.nr), device=vel.device, dtype=torch.float32)
        _numel(out, nsamp * nsg * self.nt * self.nr, "out")
        check(lib().fwi_forward(self._h, _dev_ptr(vel, torch.float32, "vel"), nsamp, keep[3], keep[4], keep[5], nsg,
                                _dev_ptr(out, torch.float32, "out"), _stream(stream)), "fwi_forward")
        return out

    def gradient(self, vel, perm, w, sg_sizes, d_obs, sigma, scale=0.0, grad=None, misfit=None, stream=None):
        """(misfit [nsamp] float64, grad [nsamp, *shape] float32) (fwi_gradient)."""
        torch = _torch()
        nsamp = vel.shape[0]
        keep = self._enc(nsamp, perm, w, sg_sizes)
        nsg = len(keep[2])
        _numel(vel, nsamp * self.phys, "vel")
        _numel(d_obs, self.ns * self.nt * self.nr, "d_obs")
        if grad is None:
            grad = torch.empty_like(vel)
        if misfit is None:
            misfit = torch.empty(nsamp, device=vel.device, dtype=torch.float64)
        _numel(grad, nsamp * self.phys, "grad")
        _numel(misfit, nsamp, "misfit")
        check(lib().fwi_gradient(self._h, _dev_ptr(vel, torch.float32, "vel"), nsamp, keep[3], keep[4], keep[5],
                                 nsg, _dev_ptr(d_obs, torch.float32, "d_obs"), float(sigma), float(scale),
                                 _dev_ptr(grad, torch.float32, "grad"), _dev_ptr(misfit, torch.float64, "misfit"),
                                 _stream(stream)), "fwi_gradient")
        return misfit, grad

    def adjoint(self, vel, perm, w, sg_sizes, d_cot, grad=None, stream=None):
        """Transposed Jacobian of the encoded records applied to d_cot
        [nsamp][nsg][nt][nr]: grad [nsamp, *shape] float32 (fwi_adjoint)."""
        torch = _torch()
        nsamp = vel.shape[0]
        keep = self._enc(nsamp, perm, w, sg_sizes)
        nsg = len(keep[2])
        _numel(vel, nsamp * self.phys, "vel")
        if tuple(d_cot.shape) != (nsamp, nsg, self.nt, self.nr):
            raise ValueError("d_cot must have shape %s, got %s" % ((nsamp, nsg, self.nt, self.nr), tuple(d_cot.shape)))
        if grad is None:
            grad = torch.empty_like(vel)
        _numel(grad, nsamp * self.phys, "grad")
        check(lib().fwi_adjoint(self._h, _dev_ptr(vel, torch.float32, "vel"), nsamp, keep[3], keep[4], keep[5], nsg,
                                _dev_ptr(d_cot, torch.float32, "d_cot"), _dev_ptr(grad, torch.float32, "grad"),
                                _stream(stream)), "fwi_adjoint")
        return grad

    def smooth_prior_grad(self, z, zref, lam, mu, grad, stream=None):
        """grad += gradient of the Gaussian smoothness prior (smooth_prior_grad)."""
        torch = _torch()
        _numel(z, z.shape[0] * self.phys, "z")
        _numel(zref, self.phys, "zref")
        _numel(grad, z.shape[0] * self.phys, "grad")
        check(lib().smooth_prior_grad(self._h, _dev_ptr(z, torch.float32, "z"), _dev_ptr(zref, torch.float32, "zref"),
                                      z.shape[0], float(lam), float(mu), _dev_ptr(grad, torch.float32, "grad"),
                                      _stream(stream)), "smooth_prior_grad")
        return grad

    def langevin_precond(self, z, grad, v, k, eta, nu, vmin, vmax, seed, counter, m=None, alpha=0.9, beta1=0.9,
                         eps=1e-2, stream=None):
        """In place: preconditioned Langevin (m None) or Adam (m given, nu 0)
        step on z [nsamp, *shape], moments v (and m) updated; k >= 1 is the
        step number of the bias correction (langevin_step_precond)."""
        torch = _torch()
        nsamp = z.shape[0]
        n = nsamp * self.phys
        _numel(z, n, "z")
        _numel(grad, n, "grad")
        _numel(v, n, "v")
        if m is not None:
            _numel(m, n, "m")
        check(lib().langevin_step_precond(self._h, _dev_ptr(z, torch.float32, "z"), _dev_ptr(grad, torch.float32, "grad"),
                                          _dev_ptr(v, torch.float32, "v"),
                                          _dev_ptr(m, torch.float32, "m") if m is not None else None, nsamp,
                                          float(alpha), float(beta1), float(eps), int(k), float(eta), float(nu),
                                          float(vmin), float(vmax), ctypes.c_uint64(seed), ctypes.c_uint64(counter),
                                          _stream(stream)), "langevin_step_precond")
        return z

    def plan_info(self):
        K, S, used, avail = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rec = ctypes.c_int64()
        check(lib().fwi_plan_info(self._h, ctypes.byref(K), ctypes.byref(S), ctypes.byref(rec), ctypes.byref(used),
                                  ctypes.byref(avail)), "fwi_plan_info")
        ch = ctypes.c_int()
        check(lib().fwi_chunking(self._h, ctypes.byref(ch)), "fwi_chunking")
        return {"segment_len": K.value, "segments": S.value, "recomputed_steps": rec.value,
                "slots_used": used.value, "slots_available": avail.value, "samples_per_chunk": ch.value}

    def set_variants(self, fwd=-1, adj=-1):
        """Force step-kernel variants (-1: autotune on the next call)."""
        check(lib().fwi_set_kernel_variants(self._h, int(fwd), int(adj)), "fwi_set_kernel_variants")

    def variants(self):
        f, a, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        fn, an = ctypes.c_char_p(), ctypes.c_char_p()
        fm, am = (ctypes.c_float * 32)(), (ctypes.c_float * 32)()
        check(lib().fwi_kernel_variants(self._h, ctypes.byref(f), ctypes.byref(a), ctypes.byref(fn), ctypes.byref(an),
                                        fm, am, ctypes.byref(n)), "fwi_kernel_variants")
        return {"forward": f.value, "adjoint": a.value, "forward_name": (fn.value or b"").decode(),
                "adjoint_name": (an.value or b"").decode(), "forward_ms": list(fm)[:n.value],
                "adjoint_ms": list(am)[:n.value]}

    def device_status(self, stream=None):
        return lib().fwi_last_device_status(self._h, _stream(stream))

    def set_profiling(self, on=True):
        check(lib().fwi_set_profiling(self._h, int(on)), "fwi_set_profiling")

    def phase_times(self):
        ms = (ctypes.c_float * 4)()
        ln = (ctypes.c_int64 * 4)()
        check(lib().fwi_phase_times(self._h, ms, ln), "fwi_phase_times")
        return list(ms), list(ln)


def langevin_step(z, grad, eta, nu, vmin, vmax, seed, counter, stream=None):
    """In place: z <- clamp(z - eta grad + nu xi, vmin, vmax) (langevin_step)."""
    torch = _torch()
    _numel(grad, z.numel(), "grad")
    check(lib().langevin_step(_dev_ptr(z, torch.float32, "z"), _dev_ptr(grad, torch.float32, "grad"), z.numel(),
                              float(eta), float(nu), float(vmin), float(vmax), ctypes.c_uint64(seed),
                              ctypes.c_uint64(counter), _stream(stream)), "langevin_step")
    return z


def renoise(x_t, x0, abar_t, abar_prev, beta_t, seed, counter, out=None, stream=None):
    """Draw x_{t-1} ~ N(mu~_t(x_t, x0), beta~_t I) (renoise)."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(x_t)
    _numel(x0, x_t.numel(), "x0")
    _numel(out, x_t.numel(), "out")
    check(lib().renoise(_dev_ptr(out, torch.float32, "out"), _dev_ptr(x_t, torch.float32, "x_t"),
                        _dev_ptr(x0, torch.float32, "x0"), x_t.numel(), float(abar_t), float(abar_prev), float(beta_t),
                        ctypes.c_uint64(seed), ctypes.c_uint64(counter), _stream(stream)), "renoise")
    return out


def residual_misfit_noalloc(d_pred, d_obs, perm, w, sg_sizes, sigma, scale=0.0, rhat=None, misfit=None, stream=None):
    """Encoded residual / misfit without any device allocation by the library
    (fwi_residual_misfit_noalloc): for callers that cannot allocate.  Returns
    (misfit [nsamp] float64, rhat like d_pred).  Calls overlapping on the GPU
    share one static scratch array and race."""
    torch = _torch()
    nsamp, nsg, nt, nr = d_pred.shape
    ns = d_obs.shape[0]
    perm = np.ascontiguousarray(np.broadcast_to(np.asarray(perm, np.int32), (nsamp, ns)))
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(w, np.int8), (nsamp, ns)))
    sg = np.ascontiguousarray(sg_sizes, np.int32)
    if len(sg) != nsg:
        raise ValueError("d_pred has %d supergathers, sg_sizes %d" % (nsg, len(sg)))
    _numel(d_obs, ns * nt * nr, "d_obs")
    if rhat is None:
        rhat = torch.empty_like(d_pred)
    if misfit is None:
        misfit = torch.empty(nsamp, device=d_pred.device, dtype=torch.float64)
    _numel(rhat, d_pred.numel(), "rhat")
    _numel(misfit, nsamp, "misfit")
    check(lib().fwi_residual_misfit_noalloc(
        _dev_ptr(d_pred, torch.float32, "d_pred"), _dev_ptr(d_obs, torch.float32, "d_obs"), nsamp, ns, nt, nr,
        perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
        sg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(sg), float(sigma), float(scale),
        _dev_ptr(rhat, torch.float32, "rhat"), _dev_ptr(misfit, torch.float64, "misfit"), _stream(stream)),
        "fwi_residual_misfit_noalloc")
    return misfit, rhat
