"""Learned prior g_theta (Sec. 2.2) on the tensor-core kernels.

1. The tcgen05 forward of the U-Net equals a PyTorch FP32 evaluation of the
   same network that rounds weights and activations to BF16 at the same points
   (the remaining difference is FP32 accumulation order and, rarely, a BF16
   rounding flipped by it).
2. Trained briefly on seeded geology patches (with PyTorch autograd, and
   with the library's own forward and backward kernels), the network predicts
   the clean model better than the stationary Gaussian prior's exact MMSE
   denoiser and than no prior at all, on held-out patches, over the noise
   levels the sampler visits.
"""
import math

import numpy as np
import pytest

import synth.patches as SP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2512_12797_gb300 import build
    build.build()
    from paper_2512_12797_gb300 import unet
    return unet


def test_tc_forward_matches_bf16_reference(U):
    import torch
    p = U.init_params(3, out_scale=8.0)
    g = torch.Generator().manual_seed(4)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * torch.randn(p[k].shape, generator=g).cuda()
    x0 = torch.tensor(SP.geology_patches(2, 64, 5)).cuda()
    sig = torch.tensor([0.3, 1.0]).cuda()
    y = (x0 + sig.view(-1, 1, 1) * torch.randn(x0.shape, generator=g).cuda()).contiguous()
    rnd = lambda t: t.to(torch.bfloat16).float()
    pb = {k: (rnd(v) if k.endswith(".w") else v) for k, v in p.items()}
    ref = U.forward_torch(pb, y, sig, act_round=rnd)
    out = U.forward_tc(U.pack(p), y, sig)
    r = float((out - ref).norm() / (ref - y).norm())
    assert r < 2e-2, r
    r32 = float((out - U.forward_torch(p, y, sig)).norm() / (ref - y).norm())
    assert r32 < 0.1, r32


def test_trained_prior_beats_gaussian_and_no_prior(U):
    import torch
    from paper_2512_12797_gb300.sampler import GaussianPriorDenoiser
    train_set = torch.tensor(SP.geology_patches(8192, 64, 11)).cuda()
    p = U.init_params(0)
    hist = U.train(p, train_set, steps=800, batch=64, lr=2e-3, seed=1, log_every=100, backend="torch")
    assert hist[-1] < hist[0]
    held = torch.tensor(SP.geology_patches(256, 64, 99)).cuda()
    den = U.UNetDenoiser(p)
    mean = torch.full((64, 64), float(train_set.mean()), device="cuda")
    gauss = GaussianPriorDenoiser(mean, corr_cells=6.0, amp=float(train_set.std()))
    g = torch.Generator(device="cuda").manual_seed(7)
    for sigma in (0.2, 0.5, 1.0):
        abar = 1.0 / (1.0 + sigma * sigma)
        x_t = math.sqrt(abar) * (held + sigma * torch.randn(held.shape, device="cuda", generator=g))
        e_unet = float(((den(x_t, abar) - held) ** 2).mean())
        e_gauss = float(((gauss(x_t, abar) - held) ** 2).mean())
        assert e_unet < 0.7 * e_gauss, (sigma, e_unet, e_gauss)
        assert e_unet < 0.3 * sigma * sigma, (sigma, e_unet)


def test_tc_backward_matches_autograd(U):
    # Gradients of sum(g * x0-hat) on the tcgen05 kernels against autograd of
    # the BF16-rounding reference.  The two forwards already differ by ~1e-2
    # (accumulation order, and the BF16 roundings and ReLU decisions that it
    # flips); ten layers of backpropagation amplify that, most in the bias
    # gradients (sums over all pixels with heavy cancellation).  Agreement is
    # therefore a few percent in norm with the direction kept (cosine > 0.99),
    # while a wiring mistake (channel split, skip, pooling adjoint) shows up as
    # an O(1) error.  The kernels themselves are checked against the FP64
    # oracle in test_gpu_prior.
    import torch
    p = U.init_params(5, out_scale=8.0)
    gen = torch.Generator().manual_seed(6)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * torch.randn(p[k].shape, generator=gen).cuda()
    x0 = torch.tensor(SP.geology_patches(4, 64, 7)).cuda()
    sig = torch.tensor([0.1, 0.3, 0.7, 1.5]).cuda()
    y = (x0 + sig.view(-1, 1, 1) * torch.randn(x0.shape, generator=gen).cuda()).contiguous()
    g = torch.randn(y.shape, generator=gen).cuda()
    rnd = lambda t: t.to(torch.bfloat16).float()
    pb = {k: (rnd(v) if k.endswith(".w") else v).clone().requires_grad_(True) for k, v in p.items()}
    (U.forward_torch(pb, y, sig, act_round=rnd) * g).sum().backward()
    q = U.pack(p)
    _, saved = U.forward_tc_train(q, y, sig)
    grads = U.backward_tc(q, saved, g)
    worst = []
    for k, v in pb.items():
        ref = v.grad
        got = grads[k].view_as(ref)
        rel = float((got - ref).norm() / ref.norm().clamp_min(1e-30))
        cos = float((got * ref).sum() / (got.norm() * ref.norm()).clamp_min(1e-30))
        worst.append((rel, cos, k))
    print("tcgen05 backward vs autograd, worst (rel, cos, name):", max(worst), min(worst, key=lambda w: w[1]))
    for rel, cos, k in worst:
        assert rel < 0.15 and cos > 0.99, (k, rel, cos)
        if k.endswith(".w"):
            assert rel < 0.1 and cos > 0.995, (k, rel, cos)


def test_training_on_tcgen05_kernels_beats_gaussian(U):
    import torch
    from paper_2512_12797_gb300.sampler import GaussianPriorDenoiser
    train_set = torch.tensor(SP.geology_patches(8192, 64, 12)).cuda()
    p = U.init_params(1)
    hist = U.train(p, train_set, steps=800, batch=64, lr=2e-3, seed=2, log_every=100, backend="tc")
    assert hist[-1] < hist[0]
    held = torch.tensor(SP.geology_patches(256, 64, 98)).cuda()
    den = U.UNetDenoiser(p)
    mean = torch.full((64, 64), float(train_set.mean()), device="cuda")
    gauss = GaussianPriorDenoiser(mean, corr_cells=6.0, amp=float(train_set.std()))
    gen = torch.Generator(device="cuda").manual_seed(8)
    for sigma in (0.2, 0.5, 1.0):
        abar = 1.0 / (1.0 + sigma * sigma)
        x_t = math.sqrt(abar) * (held + sigma * torch.randn(held.shape, device="cuda", generator=gen))
        e_unet = float(((den(x_t, abar) - held) ** 2).mean())
        e_gauss = float(((gauss(x_t, abar) - held) ** 2).mean())
        assert e_unet < 0.7 * e_gauss, (sigma, e_unet, e_gauss)
