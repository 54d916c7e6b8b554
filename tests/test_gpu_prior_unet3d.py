"""Learned prior for the 3D models (Sec. 2.2; the U-Net with 3x3x3
convolutions, paper_2512_12797_gb300/unet3d.py) on the tensor-core kernels.

1. The tcgen05 forward equals a PyTorch FP32 evaluation of the same network
   that rounds weights and activations to BF16 at the same points.
2. The tcgen05 backward (data and weight gradients of every 3x3x3 layer)
   agrees with autograd of that reference, to the tolerances of the 2D
   network (its reasoning: the two forwards differ by ~1e-2 and ten layers
   amplify it; a wiring mistake is an O(1) error).
3. Trained on seeded layered-volume patches with the tcgen05 forward and
   backward, the network denoises held-out patches better than the
   stationary Gaussian prior's exact MMSE denoiser and than no prior.
"""
import math

import pytest

import synth.patches as SP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U3():
    from paper_2512_12797_gb300 import build
    build.build()
    from paper_2512_12797_gb300 import unet3d
    return unet3d


def _noisy(torch, x0, sig, gen):
    return (x0 + sig.view(-1, 1, 1, 1) * torch.randn(x0.shape, generator=gen).cuda()).contiguous()


def _params(torch, U3, seed):
    p = U3.init_params(seed, out_scale=8.0)
    gen = torch.Generator().manual_seed(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * torch.randn(p[k].shape, generator=gen).cuda()
    return p, gen


def test_tc3_forward_matches_bf16_reference(U3):
    import torch
    p, gen = _params(torch, U3, 3)
    x0 = torch.tensor(SP.volume_patches(2, 32, 5)).cuda()
    sig = torch.tensor([0.3, 1.0]).cuda()
    y = _noisy(torch, x0, sig, gen)
    rnd = lambda t: t.to(torch.bfloat16).float()
    pb = {k: (rnd(v) if k.endswith(".w") else v) for k, v in p.items()}
    ref = U3.forward_torch(pb, y, sig, act_round=rnd)
    out = U3.forward_tc(U3.pack(p), y, sig)
    r = float((out - ref).norm() / (ref - y).norm())
    assert r < 2e-2, r
    r32 = float((out - U3.forward_torch(p, y, sig)).norm() / (ref - y).norm())
    assert r32 < 0.1, r32


def test_denoiser_layout_kernels_match_reshape_path(U3):
    # UNet3DDenoiser runs the network on the layout kernels (input built and
    # padded in the first layer, pooling, upsample-and-join, output); the
    # training path builds the same tensors with PyTorch reshapes.  Same
    # BF16 activations up to the first layer's FP32 summation order.
    import math
    import torch
    import torch.nn.functional as F
    p, gen = _params(torch, U3, 4)
    x_t = torch.tensor(SP.volume_patches(2, 32, 6)).cuda()[:, 3:29, 2:30, 1:31].contiguous()  # 26 x 28 x 30
    abar = 0.6
    got = U3.UNet3DDenoiser(p)(x_t, abar)
    n, D, H, W = x_t.shape
    Dp, Hp, Wp = U3.tile_shape(D, H, W)
    y = x_t / math.sqrt(abar)
    yp = F.pad(y[:, None], (0, Wp - W, 0, Hp - H, 0, Dp - D), mode="replicate")[:, 0].contiguous()
    sig = torch.full((n,), math.sqrt((1.0 - abar) / abar), device=x_t.device)
    ref = U3.forward_tc(U3.pack(p), yp, sig)[:, :D, :H, :W]
    r = float((got - ref).norm() / (ref - y).norm())
    assert got.shape == x_t.shape and r < 1e-2, r


def test_tc3_backward_matches_autograd(U3):
    import torch
    p, gen = _params(torch, U3, 5)
    x0 = torch.tensor(SP.volume_patches(2, 32, 7)).cuda()
    sig = torch.tensor([0.2, 0.8]).cuda()
    y = _noisy(torch, x0, sig, gen)
    g = torch.randn(y.shape, generator=gen).cuda()
    rnd = lambda t: t.to(torch.bfloat16).float()
    pb = {k: (rnd(v) if k.endswith(".w") else v).clone().requires_grad_(True) for k, v in p.items()}
    (U3.forward_torch(pb, y, sig, act_round=rnd) * g).sum().backward()
    q = U3.pack(p)
    _, saved = U3.forward_tc_train(q, y, sig)
    grads = U3.backward_tc(q, saved, g)
    worst = []
    for k, v in pb.items():
        ref = v.grad
        got = grads[k].view_as(ref)
        rel = float((got - ref).norm() / ref.norm().clamp_min(1e-30))
        cos = float((got * ref).sum() / (got.norm() * ref.norm()).clamp_min(1e-30))
        worst.append((rel, cos, k))
    print("3D tcgen05 backward vs autograd, worst (rel, cos, name):", max(worst), min(worst, key=lambda w: w[1]))
    for rel, cos, k in worst:
        assert rel < 0.15 and cos > 0.99, (k, rel, cos)
        if k.endswith(".w"):
            assert rel < 0.1 and cos > 0.995, (k, rel, cos)


def test_3d_training_on_tcgen05_kernels_beats_gaussian_and_no_prior(U3):
    import torch
    from paper_2512_12797_gb300.sampler import GaussianPriorDenoiser
    train_set = torch.tensor(SP.volume_patches(2048, 32, 21)).cuda()
    p = U3.init_params(2)
    hist = U3.train(p, train_set, steps=1500, batch=8, lr=2e-3, seed=3, log_every=100, backend="tc")
    assert hist[-1] < hist[0], hist
    held = torch.tensor(SP.volume_patches(64, 32, 97)).cuda()
    den = U3.UNet3DDenoiser(p)
    mean = torch.full((32, 32, 32), float(train_set.mean()), device="cuda")
    gauss = GaussianPriorDenoiser(mean, corr_cells=6.0, amp=float(train_set.std()))
    gen = torch.Generator(device="cuda").manual_seed(9)
    res = []
    for sigma in (0.2, 0.5, 1.0):
        abar = 1.0 / (1.0 + sigma * sigma)
        x_t = math.sqrt(abar) * (held + sigma * torch.randn(held.shape, device="cuda", generator=gen))
        e_unet = float(((den(x_t, abar) - held) ** 2).mean())
        e_gauss = float(((gauss(x_t, abar) - held) ** 2).mean())
        res.append((sigma, e_unet, e_gauss))
    print("3D prior: (sigma, unet mse, gaussian mse)", res, "loss", hist)
    # Training is not bit-reproducible (the weight gradient accumulates with
    # FP32 atomics), and three runs of this recipe ended at 0.38 / 0.48 / 0.66,
    # 0.59 / 0.65 / 0.93 and 0.44 / 0.49 / 0.66 of the Gaussian's error at
    # sigma = 0.2 / 0.5 / 1.  Asserted, with margin for that spread: below
    # the Gaussian at the lower noise levels, far below no prior at all.
    for sigma, e_unet, e_gauss in res:
        assert e_unet < 0.2 * sigma * sigma, res
        if sigma <= 0.5:
            assert e_unet < 0.9 * e_gauss, res
