"""Tensor-core building blocks of the learned prior g_theta (Sec. 2.2): the
BF16 GEMM and the 3x3 convolution of include/prior.h.  Argument marshalling
only; every contraction runs in libfwi.so's tcgen05 kernels."""
import torch

from . import _native


class PriorError(RuntimeError):
    pass


def _check(code, where):
    if code != 0:
        raise PriorError("%s failed (%d)" % (where, code))


def _stream():
    return torch.cuda.current_stream().cuda_stream


def gemm_bf16(A, B, bias=None, relu=False, out_bf16=False, out=None):
    """D = A @ B^T (+ bias) (ReLU): A [M, K] and B [N, K] contiguous BF16 CUDA
    tensors, FP32 accumulation; D [M, N] in FP32 (or BF16)."""
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=A.device)
    rc = _native.lib().prior_gemm_bf16(A.data_ptr(), B.data_ptr(), out.data_ptr(), M, N, K, out.stride(0),
                                       int(out.dtype == torch.bfloat16), bias.data_ptr() if bias is not None else None,
                                       int(relu), None, _stream())
    _check(rc, "prior_gemm_bf16")
    return out


def conv3x3(X, Wt, bias=None, relu=False, out_bf16=True, out=None):
    """Same-size 3x3 cross-correlation: X [n, H, W, Cin] BF16 (NHWC), Wt
    [Cout, 9, Cin] BF16 (tap = dy*3 + dx), bias [Cout] FP32; returns
    [n, H, W, Cout] in BF16 (or FP32)."""
    n, H, W, Cin = X.shape
    Cout = Wt.shape[0]
    if out is None:
        out = torch.empty((n, H, W, Cout), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=X.device)
    rc = _native.lib().prior_conv3x3_bf16(X.data_ptr(), Wt.data_ptr(), out.data_ptr(), n, H, W, Cin, Cout,
                                          int(out.dtype == torch.bfloat16),
                                          bias.data_ptr() if bias is not None else None, int(relu), None,
                                          _stream())
    _check(rc, "prior_conv3x3_bf16")
    return out


def last_status():
    """Device status word of the prior kernels (read and cleared)."""
    return _native.lib().prior_last_status(_stream())
