"""Learned prior g_theta (Sec. 2.2): a small U-Net that predicts the clean
normalised velocity model x0 from y = x_t / sqrt(abar_t) = x0 + sigma eps,
sigma^2 = (1 - abar_t) / abar_t, given sigma (a noise-level input map).

    x0-hat = y + f(y, sigma),
    f: 3 levels (64, 128, 256 channels), two 3x3 conv + ReLU per level,
       average-pool down, nearest up, skip concatenation, 1x1 output conv.

Two evaluations of the same parameters:
  forward_torch -- plain PyTorch in FP32, used for training with autograd;
  forward_tc    -- inference on the library's kernels: every 3x3
                   convolution but the first is prior.conv3x3 on tcgen05
                   (BF16 activations, FP32 accumulation), the first (2 real
                   input channels) runs on the CUDA cores with its input
                   built on the fly, pooling and the decoder's
                   upsample-and-join are one kernel each, and the 1x1 output
                   is prior.gemm_bf16 plus one kernel for the skip to y.
The network is fully convolutional; applied to a whole model it is the
patchwise x0 prediction with overlapping patches taken to the limit (A17),
after edge-padding to a shape the kernels tile.
"""
import math

import torch
import torch.nn.functional as F

from . import prior as TC

# (name, input channels, output channels) of the 3x3 layers, in order
LAYERS = [("e1a", 2, 64), ("e1b", 64, 64), ("e2a", 64, 128), ("e2b", 128, 128), ("ba", 128, 256),
          ("bb", 256, 256), ("d2a", 384, 128), ("d2b", 128, 128), ("d1a", 192, 64), ("d1b", 64, 64)]


def init_params(seed, device="cuda", out_scale=0.0):
    """He-initialised 3x3 layers, zero biases, and a 1x1 output layer scaled by
    out_scale (0: the untrained network is the identity x0-hat = y)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = (torch.randn(cout, cin, 3, 3, generator=g) * math.sqrt(2.0 / (9 * cin))).to(device)
        p[name + ".b"] = torch.zeros(cout, device=device)
    p["out.w"] = (torch.randn(1, 64, 1, 1, generator=g) * out_scale / 8.0).to(device)
    p["out.b"] = torch.zeros(1, device=device)
    return p


def forward_torch(p, y, sigma, act_round=None):
    """Reference forward: y [n, H, W], sigma [n] -> x0-hat [n, H, W] (FP32).
    act_round (e.g. a BF16 round trip) is applied to every conv output, to
    mimic the tcgen05 path's rounding points."""
    rnd = act_round or (lambda t: t)
    x = y[:, None]
    h = torch.cat([x, sigma.view(-1, 1, 1, 1).expand_as(x)], 1)

    def c(h, name):
        return rnd(F.relu(F.conv2d(h, p[name + ".w"], p[name + ".b"], padding=1)))

    h = c(h if act_round is None else rnd(h), "e1a")
    e1 = c(h, "e1b")
    h = c(rnd(F.avg_pool2d(e1, 2)), "e2a")
    e2 = c(h, "e2b")
    h = c(rnd(F.avg_pool2d(e2, 2)), "ba")
    h = c(h, "bb")
    h = c(torch.cat([F.interpolate(h, scale_factor=2, mode="nearest"), e2], 1), "d2a")
    h = c(h, "d2b")
    h = c(torch.cat([F.interpolate(h, scale_factor=2, mode="nearest"), e1], 1), "d1a")
    h = c(h, "d1b")
    return y + F.conv2d(h, p["out.w"], p["out.b"])[:, 0]


def pack(p):
    """Parameters in the tcgen05 layouts: 3x3 weights [Cout][9][Cin'] BF16 with
    Cin' = Cin rounded up to 64 (zero input channels), FP32 biases; the 1x1
    output as a [32][64] BF16 matrix whose row 0 is the real filter."""
    q = {}
    for name, cin, cout in LAYERS:
        w = p[name + ".w"].detach().float()
        cinp = (cin + 63) // 64 * 64
        wt = torch.zeros(cout, 9, cinp, device=w.device)
        wt[:, :, :cin] = w.permute(0, 2, 3, 1).reshape(cout, 9, cin)  # tap = dy*3 + dx
        q[name] = (wt.to(torch.bfloat16).contiguous(), p[name + ".b"].detach().float().contiguous())
    wo = torch.zeros(32, 64, device=p["out.w"].device)
    wo[0] = p["out.w"].detach().float().view(64)
    q["out"] = (wo.to(torch.bfloat16).contiguous(), float(p["out.b"].detach().float().item()))
    # the first layer's real 2 input channels, for prior_first_conv_bf16
    q["e1a2"] = (q["e1a"][0][:, :, :2].contiguous(), q["e1a"][1])
    return q


def forward_tc(q, y, sigma):
    """Inference on the library's kernels: y [n, H, W] FP32 (H, W tileable),
    sigma [n] -> x0-hat."""
    n, H, W = y.shape
    return _forward_tc(q, y, H, W, H, W, 1.0, sigma)


def _forward_tc(q, x, H, W, Hp, Wp, scale, sigma):
    """x0-hat of y = scale * x [n, H, W], evaluated on the grid edge-padded to
    Hp x Wp and cropped back: the first layer builds its 2-channel input on
    the fly (prior_first_conv_bf16), the 3x3 layers run on tcgen05, pooling
    and the decoder's upsample-and-join are single passes (prior_pool2_bf16,
    prior_upcat_bf16), and the 1x1 output is a tcgen05 GEMM whose result
    prior_output adds to y on the physical grid."""
    n = x.shape[0]

    def c(h, name):
        w, b = q[name]
        return TC.conv3x3(h, w, bias=b, relu=True)

    w2, b2 = q["e1a2"]
    h = TC.first_conv(x.contiguous(), H, W, Hp, Wp, scale, sigma.float().contiguous(), w2, b2, relu=True)
    e1 = c(h, "e1b")
    h = c(TC.pool2(e1), "e2a")
    e2 = c(h, "e2b")
    h = c(TC.pool2(e2), "ba")
    h = c(h, "bb")
    h = c(TC.upcat(h, e2), "d2a")
    h = c(h, "d2b")
    h = c(TC.upcat(h, e1), "d1a")
    h = c(h, "d1b")
    wo, bo = q["out"]
    D = TC.gemm_bf16(h.view(-1, 64), wo)
    return TC.output(D, x.contiguous(), Hp, Wp, scale, bo)


def _unpool(g):  # adjoint of the 2 x 2 average pool (NHWC)
    return (0.25 * g.float()).repeat_interleave(2, 1).repeat_interleave(2, 2)


def _downsum(g):  # adjoint of the nearest x 2 upsample (NHWC)
    n, H, W, C = g.shape
    return g.float().view(n, H // 2, 2, W // 2, 2, C).sum((2, 4))


def forward_tc_train(q, y, sigma):
    """forward_tc keeping what the backward pass needs: each conv layer's input
    and (post-ReLU) output, BF16 NHWC.  The first layer runs on tcgen05 with
    the input's 2 channels padded to a 64-channel block, so that its weight
    gradient can use the same kernel as the others."""
    n, H, W = y.shape
    x = torch.zeros((n, H, W, 64), dtype=torch.bfloat16, device=y.device)
    x[..., 0] = y.to(torch.bfloat16)
    x[..., 1] = sigma.view(n, 1, 1).to(torch.bfloat16)
    saved = {}

    def c(h, name):
        w, b = q[name]
        out = TC.conv3x3(h, w, bias=b, relu=True)
        saved[name] = (h, out)
        return out

    h = c(x, "e1a")
    e1 = c(h, "e1b")
    h = c(TC.pool2(e1), "e2a")
    e2 = c(h, "e2b")
    h = c(TC.pool2(e2), "ba")
    h = c(h, "bb")
    h = c(TC.upcat(h, e2), "d2a")
    h = c(h, "d2b")
    h = c(TC.upcat(h, e1), "d1a")
    h = c(h, "d1b")
    wo, bo = q["out"]
    o = TC.gemm_bf16(h.view(-1, 64), wo)[:, 0].view(n, H, W)
    return y + o + bo, saved


def backward_tc(q, saved, g):
    """Gradients of sum(g * x0-hat) with respect to the parameters, with every
    3x3 convolution's data and weight gradient on the tcgen05 kernels (BF16
    operands, FP32 accumulation; gradients kept in FP32 between layers).  Returns {name.w: [Cout, Cin, 3, 3],
    name.b: [Cout], out.w, out.b} in FP32, the layout of init_params."""
    grads = {}
    h = saved["d1b"][1]
    n, H, W, _ = h.shape
    gf = g.float().reshape(-1)
    wo = q["out"][0][0].float()
    grads["out.w"] = (h.view(-1, 64).float().t() @ gf).view(1, 64, 1, 1)
    grads["out.b"] = gf.sum().view(1)
    dh = g.float()[..., None] * wo  # [n, H, W, 64]

    def layer(name, d_out, need_dx=True):
        # gradients stay FP32 between layers; BF16 only as convolution operands
        x, a = saved[name]
        dzf = d_out.float() * (a > 0)  # through the ReLU
        dz = dzf.to(torch.bfloat16).contiguous()
        cin = dict((l[0], l[1]) for l in LAYERS)[name]
        grads[name + ".b"] = dzf.sum((0, 1, 2))
        dw = TC.conv3x3_wgrad(dz, x)  # [Cout, 9, Cin']
        grads[name + ".w"] = dw[:, :, :cin].reshape(dw.shape[0], 3, 3, cin).permute(0, 3, 1, 2).contiguous()
        return TC.conv3x3_dgrad(dz, q[name][0], out_bf16=False) if need_dx else None

    d = layer("d1b", dh)
    d = layer("d1a", d)                       # [.., 192] = up(d2b out) | e1
    d_up1, d_e1 = d[..., :128], d[..., 128:]
    d = layer("d2b", _downsum(d_up1))
    d = layer("d2a", d)                       # [.., 384] = up(bb out) | e2
    d_up2, d_e2 = d[..., :256], d[..., 256:]
    d = layer("bb", _downsum(d_up2))
    d = layer("ba", d)
    d_e2 = d_e2 + _unpool(d)
    d = layer("e2b", d_e2)
    d = layer("e2a", d)
    d_e1 = d_e1 + _unpool(d)
    d = layer("e1b", d_e1)
    layer("e1a", d, need_dx=False)
    return grads


def _width_ok(w):
    for lev in range(3):
        if w % (1 << lev):
            return False
        wl = w >> lev
        if not (wl % 128 == 0 or (wl <= 128 and wl & (wl - 1) == 0)):
            return False
    return True


def _shape_ok(h, w):
    return _width_ok(w) and all(h % (1 << lev) == 0 and (h >> lev) % (128 // min(w >> lev, 128)) == 0
                                for lev in range(3))


def tile_shape(H, W):
    """Smallest (H', W') >= (H, W) that the convolution kernel tiles at all
    three levels: each level's width a power of two <= 128 or a multiple of
    128, and its height a multiple of 128 / min(width, 128)."""
    Wp = W
    while not _width_ok(Wp):
        Wp += 1
    Hp = H
    while not _shape_ok(Hp, Wp):
        Hp += 1
    return Hp, Wp


def train(p, patches, steps, batch=64, lr=2e-3, sigma_range=(0.02, 3.0), seed=0, log_every=0, backend="tc"):
    """Adam on E || x0-hat(x0 + sigma eps, sigma) - x0 ||^2 with sigma
    log-uniform in sigma_range, over FP32 patches [N, S, S] on the device.
    backend "torch": PyTorch convolutions and autograd in FP32; "tc": forward
    and backward convolutions on the tcgen05 kernels (BF16 activations and
    gradients, FP32 accumulation and FP32 master weights)."""
    if backend == "tc":
        return _train_tc(p, patches, steps, batch, lr, sigma_range, seed, log_every)
    for v in p.values():
        v.requires_grad_(True)
    opt = torch.optim.Adam(list(p.values()), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    g = torch.Generator(device=patches.device).manual_seed(seed)
    lo, hi = math.log(sigma_range[0]), math.log(sigma_range[1])
    hist = []
    for k in range(steps):
        idx = torch.randint(0, patches.shape[0], (batch,), device=patches.device, generator=g)
        x0 = patches[idx]
        sig = torch.exp(lo + (hi - lo) * torch.rand(batch, device=patches.device, generator=g))
        y = x0 + sig.view(-1, 1, 1) * torch.randn(x0.shape, device=patches.device, generator=g)
        loss = F.mse_loss(forward_torch(p, y, sig), x0)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if log_every and k % log_every == 0:
            hist.append(float(loss.detach()))
    for v in p.values():
        v.requires_grad_(False)
    return hist


def _train_tc(p, patches, steps, batch, lr, sigma_range, seed, log_every):
    keys = list(p.keys())
    opt = torch.optim.Adam([p[k] for k in keys], lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    g = torch.Generator(device=patches.device).manual_seed(seed)
    lo, hi = math.log(sigma_range[0]), math.log(sigma_range[1])
    hist = []
    for k in range(steps):
        idx = torch.randint(0, patches.shape[0], (batch,), device=patches.device, generator=g)
        x0 = patches[idx]
        sig = torch.exp(lo + (hi - lo) * torch.rand(batch, device=patches.device, generator=g))
        y = (x0 + sig.view(-1, 1, 1) * torch.randn(x0.shape, device=patches.device, generator=g)).contiguous()
        q = pack(p)
        xh, saved = forward_tc_train(q, y, sig)
        r = xh - x0
        grads = backward_tc(q, saved, (2.0 / r.numel()) * r)  # d mean(r^2)
        for key in keys:
            p[key].grad = grads[key].view_as(p[key])
        opt.step()
        sched.step()
        if log_every and k % log_every == 0:
            hist.append(float((r * r).mean()))
    for key in keys:
        p[key].grad = None
    return hist


class UNetDenoiser:
    """x0-hat predictor for the sampler: (x_t [n, nz, nx], abar_t) -> x0-hat,
    in normalised units, evaluated on the tcgen05 kernels over the model
    edge-padded to a tileable shape."""

    def __init__(self, params):
        self.q = pack(params)

    def __call__(self, x_t, abar_t):
        n, H, W = x_t.shape
        sig = torch.full((n,), math.sqrt((1.0 - abar_t) / abar_t), device=x_t.device)
        Hp, Wp = tile_shape(H, W)
        return _forward_tc(self.q, x_t, H, W, Hp, Wp, 1.0 / math.sqrt(abar_t), sig)
