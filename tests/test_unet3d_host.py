"""Host-side logic of the 3D prior (no GPU): the tileable-shape search and the
adjoints of the pooling and upsampling steps used by its backward pass."""
import torch
import torch.nn.functional as F

from paper_2512_12797_gb300 import unet3d as U3


def _kernel_accepts(D, H, W):
    # the tiling rule of prior_conv3x3x3_bf16 (include/prior.h)
    if W >= 128:
        return W % 128 == 0
    if W & (W - 1):
        return False
    if H * W >= 128:
        return H % (128 // W) == 0
    return H & (H - 1) == 0 and D % (128 // (H * W)) == 0


def test_tile_shape_is_tileable_at_every_level_and_not_smaller():
    for shape in [(128, 256, 256), (32, 32, 32), (16, 16, 16), (20, 30, 40), (168, 296, 296), (7, 9, 130)]:
        Dp, Hp, Wp = U3.tile_shape(*shape)
        assert (Dp, Hp, Wp) >= tuple(shape) and Dp >= shape[0] and Hp >= shape[1] and Wp >= shape[2]
        for lev in range(3):
            assert Dp % (1 << lev) == 0 and Hp % (1 << lev) == 0 and Wp % (1 << lev) == 0
            assert _kernel_accepts(Dp >> lev, Hp >> lev, Wp >> lev), (shape, lev)
    assert U3.tile_shape(128, 256, 256) == (128, 256, 256)  # the 3D workload needs no padding


def test_pool_and_upsample_adjoints_match_autograd():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(2, 3, 4, 6, 8, generator=g, dtype=torch.float64, requires_grad=True)  # NCDHW
    gy = torch.randn(2, 3, 2, 3, 4, generator=g, dtype=torch.float64)
    F.avg_pool3d(x, 2).backward(gy)
    got = U3._unpool(gy.permute(0, 2, 3, 4, 1)).permute(0, 4, 1, 2, 3)
    assert torch.allclose(got.double(), x.grad, atol=1e-6)
    z = torch.randn(2, 3, 2, 3, 4, generator=g, dtype=torch.float64, requires_grad=True)
    gu = torch.randn(2, 3, 4, 6, 8, generator=g, dtype=torch.float64)
    F.interpolate(z, scale_factor=2, mode="nearest").backward(gu)
    got = U3._downsum(gu.permute(0, 2, 3, 4, 1)).permute(0, 4, 1, 2, 3)
    assert torch.allclose(got.double(), z.grad, atol=1e-5)  # the helpers compute in FP32
