"""Parity of the learned prior's tensor-core kernels (tcgen05 BF16 GEMM and
3x3 convolution, include/prior.h) with the FP64 oracle on the same BF16
inputs.  Products of BF16 values are exact in FP32, so the only error is FP32
accumulation: relative L2 error ~ sqrt(K) * 2^-24, bounded here by 2e-5."""
import numpy as np
import pytest

from oracle import prior_oracle as PO

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def P():
    from paper_2512_12797_gb300 import build
    build.build()
    from paper_2512_12797_gb300 import prior
    return prior


def _bf16(torch, shape, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(shape, generator=g).to(torch.bfloat16)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 64, 192), (384, 128, 1024), (256, 256, 512),
                                   (512, 384, 320)])
def test_gemm_matches_oracle(P, M, N, K):
    import torch
    A, B = _bf16(torch, (M, K), 1 + M), _bf16(torch, (N, K), 2 + N)
    D = P.gemm_bf16(A.cuda(), B.cuda())
    ref = PO.gemm(A.float().numpy(), B.float().numpy())
    assert _rel(D.cpu().double().numpy(), ref) < TOL
    assert P.last_status() == 0


def test_gemm_bias_relu_and_bf16_output(P):
    import torch
    M, N, K = 256, 64, 128
    A, B = _bf16(torch, (M, K), 5), _bf16(torch, (N, K), 6)
    bias = torch.linspace(-3, 3, N)
    D = P.gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, out_bf16=True)
    ref = np.maximum(PO.gemm(A.float().numpy(), B.float().numpy()) + bias.double().numpy(), 0.0)
    # one BF16 rounding of the output (relative 2^-9)
    assert np.allclose(D.float().cpu().numpy(), ref, rtol=2 ** -8, atol=1e-3)
    assert (D.float() >= 0).all()


@pytest.mark.parametrize("n,H,W,Cin,Cout", [(2, 16, 16, 64, 32), (1, 32, 64, 128, 64), (1, 8, 128, 64, 128),
                                            (1, 4, 256, 64, 256)])
def test_conv3x3_matches_oracle(P, n, H, W, Cin, Cout):
    import torch
    X, Wt = _bf16(torch, (n, H, W, Cin), 7 + H), _bf16(torch, (Cout, 9, Cin), 8 + Cout)
    bias = torch.randn(Cout, generator=torch.Generator().manual_seed(9))
    Y = P.conv3x3(X.cuda(), Wt.cuda(), bias=bias.cuda(), out_bf16=False)
    ref = PO.conv3x3(X.float().numpy(), Wt.float().numpy()) + bias.double().numpy()
    assert _rel(Y.cpu().double().numpy(), ref) < TOL
    # the image border (zero padding) is where a wrong shift would show
    assert _rel(Y[:, 0].cpu().double().numpy(), ref[:, 0]) < TOL
    assert _rel(Y[:, :, -1].cpu().double().numpy(), ref[:, :, -1]) < TOL


def test_rejects_unsupported_shapes(P):
    import torch
    from paper_2512_12797_gb300 import _native
    L = _native.lib()
    A = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    D = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    assert L.prior_gemm_bf16(A.data_ptr(), A.data_ptr(), D.data_ptr(), 100, 128, 64, 128, 0, None, 0, None, None) == -1
    assert L.prior_gemm_bf16(A.data_ptr(), A.data_ptr(), D.data_ptr(), 128, 48, 64, 128, 0, None, 0, None, None) == -1
    assert L.prior_gemm_bf16(A.data_ptr(), A.data_ptr(), D.data_ptr(), 128, 128, 40, 128, 0, None, 0, None, None) == -1
    X = torch.zeros((1, 16, 16, 32), dtype=torch.bfloat16, device="cuda")
    assert L.prior_conv3x3_bf16(X.data_ptr(), X.data_ptr(), D.data_ptr(), 1, 16, 16, 32, 64, 0, None, 0, None,
                                None) == -1


@pytest.mark.parametrize("n,H,W,Cin,Cout", [(2, 16, 16, 64, 64), (1, 32, 64, 192, 128), (2, 8, 16, 128, 384)])
def test_conv3x3_dgrad_matches_oracle(P, n, H, W, Cin, Cout):
    import torch
    dY, Wt = _bf16(torch, (n, H, W, Cout), 21 + H), _bf16(torch, (Cout, 9, Cin), 22 + Cin)
    dX = P.conv3x3_dgrad(dY.cuda(), Wt.cuda(), out_bf16=False)
    ref = PO.conv3x3_dgrad(dY.float().numpy(), Wt.float().numpy())
    assert _rel(dX.cpu().double().numpy(), ref) < TOL


@pytest.mark.parametrize("n,H,W,Cin,Cout", [(2, 16, 16, 64, 64), (1, 32, 32, 128, 256), (4, 8, 8, 64, 32),
                                            (1, 16, 64, 192, 128)])
def test_conv3x3_wgrad_matches_oracle(P, n, H, W, Cin, Cout):
    import torch
    dY, X = _bf16(torch, (n, H, W, Cout), 31 + W), _bf16(torch, (n, H, W, Cin), 32 + Cout)
    dW = P.conv3x3_wgrad(dY.cuda(), X.cuda())
    ref = PO.conv3x3_wgrad(dY.float().numpy(), X.float().numpy())
    assert _rel(dW.cpu().double().numpy(), ref) < 1e-4
    # the tap layout: the centre tap alone is the plain channel correlation
    assert _rel(dW[:, 4].cpu().double().numpy(), ref[:, 4]) < 1e-4
    assert P.last_status() == 0
    # per-split partial sums added in a fixed order: the same bits on every
    # call; the atomic form agrees to FP32 accumulation
    assert torch.equal(P.conv3x3_wgrad(dY.cuda(), X.cuda()), dW)
    dWa = P.conv3x3_wgrad(dY.cuda(), X.cuda(), deterministic=False)
    assert _rel(dWa.cpu().double().numpy(), ref) < 1e-4


# 3x3x3 convolution of volumes: the three tile forms (whole-width 128-voxel
# rows; TH rows of a plane; TD whole planes) and the depth border
@pytest.mark.parametrize("n,D,H,W,Cin,Cout", [(2, 4, 8, 16, 64, 64), (1, 8, 8, 8, 128, 32), (2, 16, 4, 4, 64, 128),
                                              (1, 3, 2, 128, 64, 256), (2, 16, 16, 16, 64, 64)])
def test_conv3x3x3_matches_oracle(P, n, D, H, W, Cin, Cout):
    import torch
    X, Wt = _bf16(torch, (n, D, H, W, Cin), 41 + D), _bf16(torch, (Cout, 27, Cin), 42 + Cout)
    bias = torch.randn(Cout, generator=torch.Generator().manual_seed(43))
    Y = P.conv3x3x3(X.cuda(), Wt.cuda(), bias=bias.cuda(), out_bf16=False)
    ref = PO.conv3x3x3(X.float().numpy(), Wt.float().numpy()) + bias.double().numpy()
    assert _rel(Y.cpu().double().numpy(), ref) < TOL
    for sl in [(slice(None), 0), (slice(None), -1), (slice(None), slice(None), 0),
               (slice(None), slice(None), slice(None), -1)]:
        assert _rel(Y[sl].cpu().double().numpy(), ref[sl]) < TOL, sl
    assert P.last_status() == 0


def test_conv3x3x3_rejects_untileable_shapes(P):
    import torch
    from paper_2512_12797_gb300 import _native
    L = _native.lib()
    X = torch.zeros((1, 4, 4, 4, 64), dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros((1, 4, 4, 4, 64), dtype=torch.float32, device="cuda")
    # 4 x 4 planes need 8 planes per tile: D = 4 is rejected; W = 24 is not a power of two
    assert L.prior_conv3x3x3_bf16(X.data_ptr(), X.data_ptr(), Y.data_ptr(), 1, 4, 4, 4, 64, 64, 0, None, 0, None,
                                  None) == -1
    assert L.prior_conv3x3x3_bf16(X.data_ptr(), X.data_ptr(), Y.data_ptr(), 1, 1, 16, 24, 64, 64, 0, None, 0, None,
                                  None) == -1


@pytest.mark.parametrize("n,D,H,W,Cin,Cout", [(1, 4, 8, 16, 64, 64), (2, 8, 4, 4, 128, 64)])
def test_conv3x3x3_dgrad_matches_oracle(P, n, D, H, W, Cin, Cout):
    import torch
    dY, Wt = _bf16(torch, (n, D, H, W, Cout), 51 + D), _bf16(torch, (Cout, 27, Cin), 52 + Cin)
    dX = P.conv3x3x3_dgrad(dY.cuda(), Wt.cuda(), out_bf16=False)
    ref = PO.conv3x3x3_dgrad(dY.float().numpy(), Wt.float().numpy())
    assert _rel(dX.cpu().double().numpy(), ref) < TOL


@pytest.mark.parametrize("n,D,H,W,Cin,Cout", [(1, 4, 8, 16, 64, 64), (2, 8, 8, 8, 128, 32)])
def test_conv3x3x3_wgrad_matches_oracle(P, n, D, H, W, Cin, Cout):
    import torch
    dY, X = _bf16(torch, (n, D, H, W, Cout), 61 + W), _bf16(torch, (n, D, H, W, Cin), 62 + Cout)
    dW = P.conv3x3x3_wgrad(dY.cuda(), X.cuda())
    ref = PO.conv3x3x3_wgrad(dY.float().numpy(), X.float().numpy())
    assert _rel(dW.cpu().double().numpy(), ref) < 1e-4
    assert _rel(dW[:, 13].cpu().double().numpy(), ref[:, 13]) < 1e-4  # centre tap
    assert _rel(dW[:, 0].cpu().double().numpy(), ref[:, 0]) < 1e-4    # corner tap
    assert P.last_status() == 0
    assert torch.equal(P.conv3x3x3_wgrad(dY.cuda(), X.cuda()), dW)


@pytest.mark.parametrize("n,H,W,Hp,Wp,Cout", [(2, 30, 50, 32, 64, 64), (1, 16, 16, 16, 16, 32)])
def test_first_conv_matches_oracle(P, n, H, W, Hp, Wp, Cout):
    # the network input built on the fly (scaled model, edge-padded to Hp x Wp,
    # noise-level channel; both rounded to BF16) and convolved from 2 channels
    import torch
    g = torch.Generator().manual_seed(n * 100 + H)
    x = torch.randn((n, H, W), generator=g) * 0.7
    sig = torch.tensor([0.3, 1.7][:n])
    Wt = _bf16(torch, (Cout, 9, 2), 5 + Cout)
    bias = torch.randn(Cout, generator=g) * 0.1
    scale = 1.25
    Y = P.first_conv(x.cuda(), H, W, Hp, Wp, scale, sig.cuda(), Wt.cuda(), bias.cuda(), relu=True)
    xin = np.zeros((n, Hp, Wp, 2))
    xp = np.pad((scale * x).numpy(), ((0, 0), (0, Hp - H), (0, Wp - W)), mode="edge")
    xin[..., 0] = torch.tensor(xp).float().to(torch.bfloat16).double().numpy()
    xin[..., 1] = sig.to(torch.bfloat16).double().numpy()[:, None, None]
    ref = np.maximum(PO.conv3x3(xin, Wt.float().numpy()) + bias.double().numpy(), 0.0)
    got = Y.cpu().double().numpy()
    # one BF16 rounding of the output on top of FP32 accumulation
    assert _rel(got, ref) < 4e-3
    assert np.max(np.abs(got - ref)) <= 2 ** -7 * np.max(np.abs(ref))


def test_pool_and_upcat_layout_kernels(P):
    import torch
    n, H, W, C1, C2 = 2, 8, 16, 64, 32
    X = _bf16(torch, (n, H, W, C2), 9)
    pooled = P.pool2(X.cuda()).cpu()
    ref = X.double().numpy().reshape(n, H // 2, 2, W // 2, 2, C2).mean(axis=(2, 4))
    assert np.max(np.abs(pooled.double().numpy() - ref)) <= 2 ** -8 * np.max(np.abs(ref))
    lo = _bf16(torch, (n, H // 2, W // 2, C1), 10)
    up = P.upcat(lo.cuda(), X.cuda()).cpu()
    assert torch.equal(up[..., :C1], lo.repeat_interleave(2, 1).repeat_interleave(2, 2))
    assert torch.equal(up[..., C1:], X)


@pytest.mark.parametrize("n,D,H,W,Dp,Hp,Wp,Cout", [(2, 6, 10, 14, 8, 16, 16, 64), (1, 8, 8, 8, 8, 8, 8, 32)])
def test_first_conv3d_matches_oracle(P, n, D, H, W, Dp, Hp, Wp, Cout):
    # the 3D network's input built on the fly (scaled volume, edge-padded to
    # Dp x Hp x Wp, noise-level channel; both rounded to BF16) and convolved
    # 3x3x3 from 2 channels
    import torch
    g = torch.Generator().manual_seed(n * 100 + D)
    x = torch.randn((n, D, H, W), generator=g) * 0.7
    sig = torch.tensor([0.3, 1.7][:n])
    Wt = _bf16(torch, (Cout, 27, 2), 7 + Cout)
    bias = torch.randn(Cout, generator=g) * 0.1
    scale = 0.8
    Y = P.first_conv3d(x.cuda(), D, H, W, Dp, Hp, Wp, scale, sig.cuda(), Wt.cuda(), bias.cuda(), relu=True)
    xin = np.zeros((n, Dp, Hp, Wp, 2))
    xp = np.pad((scale * x).numpy(), ((0, 0), (0, Dp - D), (0, Hp - H), (0, Wp - W)), mode="edge")
    xin[..., 0] = torch.tensor(xp).float().to(torch.bfloat16).double().numpy()
    xin[..., 1] = sig.to(torch.bfloat16).double().numpy()[:, None, None, None]
    ref = np.maximum(PO.conv3x3x3(xin, Wt.float().numpy()) + bias.double().numpy(), 0.0)
    got = Y.cpu().double().numpy()
    assert _rel(got, ref) < 4e-3
    assert np.max(np.abs(got - ref)) <= 2 ** -7 * np.max(np.abs(ref))


def test_pool_upcat_output_3d_layout_kernels(P):
    import torch
    n, D, H, W, C1, C2 = 2, 4, 8, 16, 64, 32
    X = _bf16(torch, (n, D, H, W, C2), 19)
    pooled = P.pool2_3d(X.cuda()).cpu()
    ref = X.double().numpy().reshape(n, D // 2, 2, H // 2, 2, W // 2, 2, C2).mean(axis=(2, 4, 6))
    assert np.max(np.abs(pooled.double().numpy() - ref)) <= 2 ** -8 * np.max(np.abs(ref))
    lo = _bf16(torch, (n, D // 2, H // 2, W // 2, C1), 20)
    up = P.upcat3d(lo.cuda(), X.cuda()).cpu()
    assert torch.equal(up[..., :C1], lo.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3))
    assert torch.equal(up[..., C1:], X)
    # output on the physical part of a padded volume, D a column of rows of 32 floats
    Dp, Hp, Wp = D + 2, H + 3, W + 4
    g = torch.Generator().manual_seed(21)
    x = torch.randn((n, D, H, W), generator=g)
    Dm = torch.randn((n * Dp * Hp * Wp, 32), generator=g)
    out = P.output3d(Dm.cuda(), x.cuda(), Dp, Hp, Wp, 1.5, 0.25).cpu()
    ref = 1.5 * x + Dm[:, 0].view(n, Dp, Hp, Wp)[:, :D, :H, :W] + 0.25
    assert torch.allclose(out, ref, rtol=1e-6, atol=1e-6)
