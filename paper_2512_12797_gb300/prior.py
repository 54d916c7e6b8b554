"""Tensor-core building blocks of the learned prior g_theta (Sec. 2.2): the
BF16 GEMM and the 3x3 and 3x3x3 convolutions of include/prior.h.  Argument marshalling
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


def first_conv(x, H, W, Hp, Wp, scale, sigma, Wt2, bias, relu=True):
    """First layer: the 2-channel network input (scale * x edge-padded to
    Hp x Wp, and sigma per image), 3x3 convolution with Wt2 [Cout][9][2] BF16
    (prior_first_conv_bf16); returns [n, Hp, Wp, Cout] BF16."""
    n = x.shape[0]
    Cout = Wt2.shape[0]
    out = torch.empty((n, Hp, Wp, Cout), dtype=torch.bfloat16, device=x.device)
    rc = _native.lib().prior_first_conv_bf16(x.data_ptr(), n, H, W, Hp, Wp, float(scale), sigma.data_ptr(),
                                             Wt2.data_ptr(), bias.data_ptr() if bias is not None else None, Cout,
                                             int(relu), out.data_ptr(), _stream())
    _check(rc, "prior_first_conv_bf16")
    return out


def pool2(X):
    """2 x 2 average pooling of X [n, H, W, C] BF16 (prior_pool2_bf16)."""
    n, H, W, C = X.shape
    out = torch.empty((n, H // 2, W // 2, C), dtype=torch.bfloat16, device=X.device)
    _check(_native.lib().prior_pool2_bf16(X.data_ptr(), n, H, W, C, out.data_ptr(), _stream()), "prior_pool2_bf16")
    return out


def upcat(lo, skip):
    """[up2(lo), skip] along channels: lo [n, H/2, W/2, C1], skip [n, H, W, C2] (prior_upcat_bf16)."""
    n, H, W, C2 = skip.shape
    C1 = lo.shape[-1]
    out = torch.empty((n, H, W, C1 + C2), dtype=torch.bfloat16, device=skip.device)
    _check(_native.lib().prior_upcat_bf16(lo.data_ptr(), C1, skip.data_ptr(), C2, n, H, W, out.data_ptr(),
                                          _stream()), "prior_upcat_bf16")
    return out


def output(D, x, Hp, Wp, scale, bo):
    """x0-hat = scale * x + D[:, 0] + bo on the physical part [n, H, W] of the
    padded grid (prior_output); D [n*Hp*Wp, ldd] FP32."""
    n, H, W = x.shape
    out = torch.empty_like(x)
    _check(_native.lib().prior_output(D.data_ptr(), D.stride(0), x.data_ptr(), n, H, W, Hp, Wp, float(scale),
                                      float(bo), out.data_ptr(), _stream()), "prior_output")
    return out


def first_conv3d(x, D, H, W, Dp, Hp, Wp, scale, sigma, Wt2, bias, relu=True):
    """First layer of the 3D network: the 2-channel input (scale * x [n, D, H, W]
    edge-padded to Dp x Hp x Wp, and sigma per volume), 3x3x3 convolution with
    Wt2 [Cout][27][2] BF16 (prior_first_conv3d_bf16); returns [n, Dp, Hp, Wp, Cout] BF16."""
    n = x.shape[0]
    Cout = Wt2.shape[0]
    out = torch.empty((n, Dp, Hp, Wp, Cout), dtype=torch.bfloat16, device=x.device)
    rc = _native.lib().prior_first_conv3d_bf16(x.data_ptr(), n, D, H, W, Dp, Hp, Wp, float(scale), sigma.data_ptr(),
                                               Wt2.data_ptr(), bias.data_ptr() if bias is not None else None, Cout,
                                               int(relu), out.data_ptr(), _stream())
    _check(rc, "prior_first_conv3d_bf16")
    return out


def pool2_3d(X):
    """2 x 2 x 2 average pooling of X [n, D, H, W, C] BF16 (prior_pool2_3d_bf16)."""
    n, D, H, W, C = X.shape
    out = torch.empty((n, D // 2, H // 2, W // 2, C), dtype=torch.bfloat16, device=X.device)
    _check(_native.lib().prior_pool2_3d_bf16(X.data_ptr(), n, D, H, W, C, out.data_ptr(), _stream()),
           "prior_pool2_3d_bf16")
    return out


def upcat3d(lo, skip):
    """[up2(lo), skip] along channels: lo [n, D/2, H/2, W/2, C1], skip [n, D, H, W, C2] (prior_upcat3d_bf16)."""
    n, D, H, W, C2 = skip.shape
    C1 = lo.shape[-1]
    out = torch.empty((n, D, H, W, C1 + C2), dtype=torch.bfloat16, device=skip.device)
    _check(_native.lib().prior_upcat3d_bf16(lo.data_ptr(), C1, skip.data_ptr(), C2, n, D, H, W, out.data_ptr(),
                                            _stream()), "prior_upcat3d_bf16")
    return out


def output3d(Dm, x, Dp, Hp, Wp, scale, bo):
    """x0-hat = scale * x + Dm[:, 0] + bo on the physical part [n, D, H, W] of the
    padded volume (prior_output3d); Dm [n*Dp*Hp*Wp, ldd] FP32."""
    n, D, H, W = x.shape
    out = torch.empty_like(x)
    _check(_native.lib().prior_output3d(Dm.data_ptr(), Dm.stride(0), x.data_ptr(), n, D, H, W, Dp, Hp, Wp,
                                        float(scale), float(bo), out.data_ptr(), _stream()), "prior_output3d")
    return out


def last_status():
    """Device status word of the prior kernels (read and cleared)."""
    return _native.lib().prior_last_status(_stream())


def flip_weights(Wt):
    """Weights of the data gradient: Wt'[c][T - 1 - t][o] = Wt[o][t][c], T = 9 or 27 taps."""
    return Wt.flip(1).transpose(0, 2).contiguous()


def conv3x3_dgrad(dY, Wt, out_bf16=True):
    """Gradient of conv3x3 with respect to its input: the same-size
    convolution of dY [n, H, W, Cout] with the flipped, transposed weights."""
    return conv3x3(dY, flip_weights(Wt), out_bf16=out_bf16)


def shifted_taps(X):
    """[9][Cin][P] BF16: X [n, H, W, Cin] shifted by (dy - 1, dx - 1) for each
    tap t = dy*3 + dx, zero off the image, channel-major over pixels P = n*H*W."""
    n, H, W, C = X.shape
    Xp = torch.nn.functional.pad(X.permute(3, 0, 1, 2), (1, 1, 1, 1))  # [C, n, H+2, W+2]
    out = torch.empty((9, C, n * H * W), dtype=X.dtype, device=X.device)
    for dy in range(3):
        for dx in range(3):
            out[dy * 3 + dx] = Xp[:, :, dy:dy + H, dx:dx + W].reshape(C, -1)
    return out


def _sms(dev):
    return torch.cuda.get_device_properties(dev).multi_processor_count


def conv3x3_wgrad(dY, X, splits=None, out=None, deterministic=True):
    """Gradient of conv3x3 with respect to its weights: dW [Cout, 9, Cin] FP32
    from the output gradient dY [n, H, W, Cout] and the input X [n, H, W, Cin].
    deterministic: per-split partial sums added in a fixed order (same result
    on every run); else FP32 atomics."""
    n, H, W, Cout = dY.shape
    Cin = X.shape[-1]
    P = n * H * W
    mp = (Cout + 127) // 128 * 128
    dYt = torch.zeros((mp, P), dtype=torch.bfloat16, device=dY.device)
    dYt[:Cout] = dY.reshape(P, Cout).t()
    X9 = shifted_taps(X.to(torch.bfloat16))
    if out is None:
        out = torch.zeros((Cout, 9, Cin), dtype=torch.float32, device=dY.device)
    if splits is None:  # about two CTAs per SM over the (co, ci, tap) tiles
        bn = Cin if Cin in (32, 64, 128, 256) else (128 if Cin % 128 == 0 else 64)
        tiles = ((Cout + 127) // 128) * (Cin // bn) * 9
        splits = max(1, min(P // 64, (2 * _sms(dY.device)) // tiles))
    work = torch.empty(splits * Cout * 9 * Cin, dtype=torch.float32, device=dY.device) if deterministic else None
    rc = _native.lib().prior_conv3x3_wgrad_bf16(dYt.data_ptr(), X9.data_ptr(), out.data_ptr(),
                                                work.data_ptr() if work is not None else None, P, Cout, Cin,
                                                splits, None, _stream())
    _check(rc, "prior_conv3x3_wgrad_bf16")
    return out


def conv3x3x3(X, Wt, bias=None, relu=False, out_bf16=True, out=None):
    """Same-size 3x3x3 cross-correlation of volumes: X [n, D, H, W, Cin] BF16
    (NDHWC), Wt [Cout, 27, Cin] BF16 (tap = dz*9 + dy*3 + dx), bias [Cout]
    FP32; returns [n, D, H, W, Cout] in BF16 (or FP32)."""
    n, D, H, W, Cin = X.shape
    Cout = Wt.shape[0]
    if out is None:
        out = torch.empty((n, D, H, W, Cout), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=X.device)
    rc = _native.lib().prior_conv3x3x3_bf16(X.data_ptr(), Wt.data_ptr(), out.data_ptr(), n, D, H, W, Cin, Cout,
                                            int(out.dtype == torch.bfloat16),
                                            bias.data_ptr() if bias is not None else None, int(relu), None,
                                            _stream())
    _check(rc, "prior_conv3x3x3_bf16")
    return out


def conv3x3x3_dgrad(dY, Wt, out_bf16=True):
    """Gradient of conv3x3x3 with respect to its input: the same-size
    convolution of dY with the flipped, transposed weights (flipping the tap
    index t = dz*9 + dy*3 + dx reverses all three offsets)."""
    return conv3x3x3(dY, flip_weights(Wt), out_bf16=out_bf16)


def shifted_taps3(X):
    """[27][Cin][P] BF16: X [n, D, H, W, Cin] shifted by (dz - 1, dy - 1, dx - 1)
    for each tap t = dz*9 + dy*3 + dx, zero off the volume, channel-major over
    voxels P = n*D*H*W."""
    n, D, H, W, C = X.shape
    Xp = torch.nn.functional.pad(X.permute(4, 0, 1, 2, 3), (1, 1, 1, 1, 1, 1))  # [C, n, D+2, H+2, W+2]
    out = torch.empty((27, C, n * D * H * W), dtype=X.dtype, device=X.device)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out[dz * 9 + dy * 3 + dx] = Xp[:, :, dz:dz + D, dy:dy + H, dx:dx + W].reshape(C, -1)
    return out


def conv3x3x3_wgrad(dY, X, splits=None, out=None, deterministic=True):
    """Gradient of conv3x3x3 with respect to its weights: dW [Cout, 27, Cin]
    FP32 from the output gradient dY [n, D, H, W, Cout] and the input X
    (deterministic as in conv3x3_wgrad)."""
    Cout = dY.shape[-1]
    Cin = X.shape[-1]
    P = dY.numel() // Cout
    mp = (Cout + 127) // 128 * 128
    dYt = torch.zeros((mp, P), dtype=torch.bfloat16, device=dY.device)
    dYt[:Cout] = dY.reshape(P, Cout).t()
    X27 = shifted_taps3(X.to(torch.bfloat16))
    if out is None:
        out = torch.zeros((Cout, 27, Cin), dtype=torch.float32, device=dY.device)
    if splits is None:  # about two CTAs per SM over the (co, ci, tap) tiles
        bn = Cin if Cin in (32, 64, 128, 256) else (128 if Cin % 128 == 0 else 64)
        tiles = ((Cout + 127) // 128) * (Cin // bn) * 27
        splits = max(1, min(P // 64, (2 * _sms(dY.device)) // tiles))
    work = torch.empty(splits * Cout * 27 * Cin, dtype=torch.float32, device=dY.device) if deterministic else None
    rc = _native.lib().prior_conv3x3x3_wgrad_bf16(dYt.data_ptr(), X27.data_ptr(), out.data_ptr(),
                                                  work.data_ptr() if work is not None else None, P, Cout, Cin,
                                                  splits, None, _stream())
    _check(rc, "prior_conv3x3x3_wgrad_bf16")
    return out


def _main():
    """Times one convolution: python -m paper_2512_12797_gb300.prior [n H W Cin Cout]
    (3x3) or [n D H W Cin Cout] (3x3x3)."""
    import sys
    from . import build
    build.build()
    a = [int(v) for v in sys.argv[1:]]
    if len(a) == 6:
        n, D, H, W, Cin, Cout = a
        X = torch.randn(n, D, H, W, Cin, device="cuda").to(torch.bfloat16)
        Wt = torch.randn(Cout, 27, Cin, device="cuda").to(torch.bfloat16)
        Y = torch.empty(n, D, H, W, Cout, device="cuda", dtype=torch.bfloat16)
        run, taps, name = (lambda: conv3x3x3(X, Wt, out=Y)), 27, "conv3x3x3 [%d, %d, %d, %d, %d]" % (n, D, H, W, Cin)
        vox = n * D * H * W
    else:
        n, H, W, Cin, Cout = a if len(a) == 5 else (16, 128, 128, 128, 128)
        X = torch.randn(n, H, W, Cin, device="cuda").to(torch.bfloat16)
        Wt = torch.randn(Cout, 9, Cin, device="cuda").to(torch.bfloat16)
        Y = torch.empty(n, H, W, Cout, device="cuda", dtype=torch.bfloat16)
        run, taps, name = (lambda: conv3x3(X, Wt, out=Y)), 9, "conv3x3 [%d, %d, %d, %d]" % (n, H, W, Cin)
        vox = n * H * W
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    flops = 2.0 * vox * taps * Cin * Cout
    print("%s -> %d: %.3f ms, %.0f TFLOP/s, status %d" % (name, Cout, ms, flops / ms / 1e9, last_status()))


if __name__ == "__main__":
    _main()
