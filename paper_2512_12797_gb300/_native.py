"""ctypes declarations of the C ABI in include/fwi.h and include/prior.h
(argument marshalling only).

Loading fails loudly when libfwi.so is missing: there is no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfwi.so")

FWI_STATUS = {0: "FWI_OK", -1: "FWI_ERR_ARG", -2: "FWI_ERR_CFL", -3: "FWI_ERR_OOM", -4: "FWI_ERR_CUDA",
              -5: "FWI_ERR_NONFINITE", -6: "FWI_ERR_TIMEOUT", -7: "FWI_ERR_BOUNDS"}

# every symbol fwi.h declares
EXPORTS = ["fwi_create", "fwi_destroy", "fwi_encode", "fwi_forward", "fwi_gradient", "fwi_adjoint", "langevin_step",
           "langevin_step_precond", "renoise",
           "smooth_prior_grad", "fwi_status_string", "fwi_last_device_status", "fwi_plan_info",
           "fwi_set_profiling", "fwi_phase_times", "fwi_residual_misfit_noalloc", "fwi_last_cuda_error",
           "fwi_set_kernel_variants", "fwi_kernel_variants", "fwi_chunking", "fwi_checkpoint_schedule"]
# every symbol prior.h declares
PRIOR_EXPORTS = ["prior_gemm_bf16", "prior_conv3x3_bf16", "prior_conv3x3_wgrad_bf16", "prior_conv3x3x3_bf16",
                 "prior_conv3x3x3_wgrad_bf16", "prior_last_status", "prior_first_conv_bf16", "prior_pool2_bf16",
                 "prior_upcat_bf16", "prior_output", "prior_first_conv3d_bf16", "prior_pool2_3d_bf16",
                 "prior_upcat3d_bf16", "prior_output3d"]


class FwiGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
                ("hz", ctypes.c_double), ("hy", ctypes.c_double), ("hx", ctypes.c_double),
                ("nb", ctypes.c_int), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
                ("f0", ctypes.c_double), ("t0", ctypes.c_double),
                ("sponge_vmax", ctypes.c_double), ("sponge_R", ctypes.c_double)]


class FwiGeom(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("src", ctypes.POINTER(ctypes.c_int32)),
                ("nr", ctypes.c_int), ("rec", ctypes.POINTER(ctypes.c_int32))]


class FwiError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, FWI_STATUS.get(code, "?"), code))


_lib = None

_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_I8P = ctypes.POINTER(ctypes.c_int8)
_SIGS = {
    "fwi_create": (ctypes.c_int, [ctypes.POINTER(FwiGrid), ctypes.POINTER(FwiGeom), ctypes.c_int, ctypes.c_size_t,
                                  ctypes.POINTER(_P)]),
    "fwi_destroy": (None, [_P]),
    "fwi_encode": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _I32P, _I8P]),
    "fwi_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _I32P, _I8P, _I32P, ctypes.c_int, _P, _P]),
    "fwi_gradient": (ctypes.c_int, [_P, _P, ctypes.c_int, _I32P, _I8P, _I32P, ctypes.c_int, _P, ctypes.c_double,
                                    ctypes.c_double, _P, _P, _P]),
    "fwi_checkpoint_schedule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _I32P, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int)]),
    "fwi_adjoint": (ctypes.c_int, [_P, _P, ctypes.c_int, _I32P, _I8P, _I32P, ctypes.c_int, _P, _P, _P]),
    "langevin_step": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, _P]),
    "langevin_step_precond": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, _P]),
    "renoise": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint64, _P]),
    "smooth_prior_grad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P]),
    "fwi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fwi_last_cuda_error": (ctypes.c_char_p, []),
    "fwi_set_kernel_variants": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "fwi_chunking": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "fwi_kernel_variants": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_char_p),
                                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_int)]),
    "fwi_last_device_status": (ctypes.c_int, [_P, _P]),
    "fwi_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "fwi_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "fwi_phase_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64)]),
    "fwi_residual_misfit_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   _I32P, _I8P, _I32P, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, _P, _P, _P]),
    "prior_gemm_bf16": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "prior_conv3x3_bf16": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "prior_conv3x3_wgrad_bf16": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _P, _P]),
    "prior_conv3x3x3_bf16": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P]),
    "prior_conv3x3x3_wgrad_bf16": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _P, _P]),
    "prior_last_status": (ctypes.c_int, [_P]),
    "prior_first_conv_bf16": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_float, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                             _P, _P]),
    "prior_pool2_bf16": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "prior_upcat_bf16": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _P, _P]),
    "prior_output": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_float, ctypes.c_float, _P, _P]),
    "prior_first_conv3d_bf16": (ctypes.c_int, [_P] + [ctypes.c_int] * 7 + [ctypes.c_float, _P, _P, _P, ctypes.c_int,
                                                                          ctypes.c_int, _P, _P]),
    "prior_pool2_3d_bf16": (ctypes.c_int, [_P] + [ctypes.c_int] * 5 + [_P, _P]),
    "prior_upcat3d_bf16": (ctypes.c_int, [_P, ctypes.c_int, _P] + [ctypes.c_int] * 5 + [_P, _P]),
    "prior_output3d": (ctypes.c_int, [_P, ctypes.c_int, _P] + [ctypes.c_int] * 7 + [ctypes.c_float, ctypes.c_float,
                                                                                    _P, _P]),
}


def lib():
    """The loaded library; raises if libfwi.so has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfwi.so not built (run paper_2512_12797_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != 0:
        if code == -4:
            where = "%s [%s]" % (where, lib().fwi_last_cuda_error().decode())
        raise FwiError(code, where)
    return code
