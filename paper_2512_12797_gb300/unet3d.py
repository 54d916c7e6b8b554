"""Learned prior g_theta (Sec. 2.2) for 3D models: the U-Net of unet.py with
3x3x3 convolutions, for volume patches of the 3D velocity models.

    x0-hat = y + f(y, sigma),   y = x_t / sqrt(abar_t) = x0 + sigma eps,
    f: 3 levels (64, 128, 256 channels), two 3x3x3 conv + ReLU per level,
       2x2x2 average-pool down, nearest up, skip concatenation, 1x1x1 output.

forward_torch  -- plain PyTorch FP32 (training with autograd, reference);
forward_tc     -- every 3x3x3 convolution on prior.conv3x3x3 (tcgen05, BF16
                  activations, FP32 accumulation), the 1x1x1 output on
                  prior.gemm_bf16; pooling, upsampling, concatenation are
                  tensor reshapes (the training path, which keeps each
                  layer's input for the backward);
_forward_tc    -- the inference path of UNet3DDenoiser: the same network with
                  the input build, padding, pooling, upsample-and-join and
                  output on the layout kernels of prior.py;
backward_tc    -- data and weight gradients of every 3x3x3 convolution on the
                  tcgen05 kernels (gradients FP32 between layers).
"""
import math

import torch
import torch.nn.functional as F

from . import prior as TC
from .unet import LAYERS


def init_params(seed, device="cuda", out_scale=0.0):
    """He-initialised 3x3x3 layers, zero biases, and a 1x1x1 output scaled by
    out_scale (0: the untrained network is the identity x0-hat = y)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = (torch.randn(cout, cin, 3, 3, 3, generator=g) * math.sqrt(2.0 / (27 * cin))).to(device)
        p[name + ".b"] = torch.zeros(cout, device=device)
    p["out.w"] = (torch.randn(1, 64, 1, 1, 1, generator=g) * out_scale / 8.0).to(device)
    p["out.b"] = torch.zeros(1, device=device)
    return p


def forward_torch(p, y, sigma, act_round=None):
    """Reference forward: y [n, D, H, W], sigma [n] -> x0-hat (FP32); act_round
    is applied where the tcgen05 path rounds to BF16."""
    rnd = act_round or (lambda t: t)
    x = y[:, None]
    h = torch.cat([x, sigma.view(-1, 1, 1, 1, 1).expand_as(x)], 1)

    def c(h, name):
        return rnd(F.relu(F.conv3d(h, p[name + ".w"], p[name + ".b"], padding=1)))

    h = c(h if act_round is None else rnd(h), "e1a")
    e1 = c(h, "e1b")
    h = c(rnd(F.avg_pool3d(e1, 2)), "e2a")
    e2 = c(h, "e2b")
    h = c(rnd(F.avg_pool3d(e2, 2)), "ba")
    h = c(h, "bb")
    h = c(torch.cat([F.interpolate(h, scale_factor=2, mode="nearest"), e2], 1), "d2a")
    h = c(h, "d2b")
    h = c(torch.cat([F.interpolate(h, scale_factor=2, mode="nearest"), e1], 1), "d1a")
    h = c(h, "d1b")
    return y + F.conv3d(h, p["out.w"], p["out.b"])[:, 0]


def pack(p):
    """tcgen05 layouts: 3x3x3 weights [Cout][27][Cin'] BF16 (tap = dz*9 + dy*3
    + dx, Cin' = Cin rounded up to 64), FP32 biases, 1x1x1 output as [32][64]."""
    q = {}
    for name, cin, cout in LAYERS:
        w = p[name + ".w"].detach().float()
        cinp = (cin + 63) // 64 * 64
        wt = torch.zeros(cout, 27, cinp, device=w.device)
        wt[:, :, :cin] = w.permute(0, 2, 3, 4, 1).reshape(cout, 27, cin)
        q[name] = (wt.to(torch.bfloat16).contiguous(), p[name + ".b"].detach().float().contiguous())
    wo = torch.zeros(32, 64, device=p["out.w"].device)
    wo[0] = p["out.w"].detach().float().view(64)
    q["out"] = (wo.to(torch.bfloat16).contiguous(), float(p["out.b"].detach().float().item()))
    q["e1a2"] = (q["e1a"][0][:, :, :2].contiguous(), q["e1a"][1])  # first layer's 2 real input channels
    return q


def _pool(h):  # NDHWC average pool 2 x 2 x 2
    n, D, H, W, C = h.shape
    return h.float().view(n, D // 2, 2, H // 2, 2, W // 2, 2, C).mean((2, 4, 6)).to(torch.bfloat16).contiguous()


def _up(h):  # NDHWC nearest upsample x 2
    return h.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def _unpool(g):  # adjoint of the average pool
    return (0.125 * g.float()).repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def _downsum(g):  # adjoint of the nearest upsample
    n, D, H, W, C = g.shape
    return g.float().view(n, D // 2, 2, H // 2, 2, W // 2, 2, C).sum((2, 4, 6))


def _input(y, sigma):
    n, D, H, W = y.shape
    x = torch.zeros((n, D, H, W, 64), dtype=torch.bfloat16, device=y.device)
    x[..., 0] = y.to(torch.bfloat16)
    x[..., 1] = sigma.view(n, 1, 1, 1).to(torch.bfloat16)
    return x


def forward_tc_train(q, y, sigma):
    """Inference on the tcgen05 kernels, y [n, D, H, W] FP32, sigma [n];
    returns x0-hat and each conv layer's (input, post-ReLU output)."""
    n, D, H, W = y.shape
    saved = {}

    def c(h, name):
        w, b = q[name]
        out = TC.conv3x3x3(h, w, bias=b, relu=True)
        saved[name] = (h, out)
        return out

    h = c(_input(y, sigma), "e1a")
    e1 = c(h, "e1b")
    h = c(_pool(e1), "e2a")
    e2 = c(h, "e2b")
    h = c(_pool(e2), "ba")
    h = c(h, "bb")
    h = c(torch.cat([_up(h), e2], -1).contiguous(), "d2a")
    h = c(h, "d2b")
    h = c(torch.cat([_up(h), e1], -1).contiguous(), "d1a")
    h = c(h, "d1b")
    wo, bo = q["out"]
    o = TC.gemm_bf16(h.view(-1, 64), wo)[:, 0].view(n, D, H, W)
    return y + o + bo, saved


def forward_tc(q, y, sigma):
    return forward_tc_train(q, y, sigma)[0]


def _forward_tc(q, x, D, H, W, Dp, Hp, Wp, scale, sigma):
    """x0-hat of y = scale * x [n, D, H, W], evaluated on the volume
    edge-padded to Dp x Hp x Wp and cropped back, with no PyTorch reshapes
    between the kernels: the first layer builds its 2-channel input on the fly
    (prior_first_conv3d_bf16), the 3x3x3 layers run on tcgen05, pooling and
    the decoder's upsample-and-join are single passes (prior_pool2_3d_bf16,
    prior_upcat3d_bf16), and the 1x1x1 output is a tcgen05 GEMM whose result
    prior_output3d adds to y on the physical volume."""
    def c(h, name):
        w, b = q[name]
        return TC.conv3x3x3(h, w, bias=b, relu=True)

    w2, b2 = q["e1a2"]
    h = TC.first_conv3d(x.contiguous(), D, H, W, Dp, Hp, Wp, scale, sigma.float().contiguous(), w2, b2, relu=True)
    e1 = c(h, "e1b")
    h = c(TC.pool2_3d(e1), "e2a")
    e2 = c(h, "e2b")
    h = c(TC.pool2_3d(e2), "ba")
    h = c(h, "bb")
    h = c(TC.upcat3d(h, e2), "d2a")
    h = c(h, "d2b")
    h = c(TC.upcat3d(h, e1), "d1a")
    h = c(h, "d1b")
    wo, bo = q["out"]
    Dm = TC.gemm_bf16(h.view(-1, 64), wo)
    return TC.output3d(Dm, x.contiguous(), Dp, Hp, Wp, scale, bo)


def backward_tc(q, saved, g):
    """Gradients of sum(g * x0-hat) with respect to the parameters (layout of
    init_params), every 3x3x3 data and weight gradient on the tcgen05 kernels."""
    grads = {}
    h = saved["d1b"][1]
    gf = g.float().reshape(-1)
    wo = q["out"][0][0].float()
    grads["out.w"] = (h.view(-1, 64).float().t() @ gf).view(1, 64, 1, 1, 1)
    grads["out.b"] = gf.sum().view(1)
    dh = g.float()[..., None] * wo
    cins = dict((l[0], l[1]) for l in LAYERS)

    def layer(name, d_out, need_dx=True):
        x, a = saved[name]
        dzf = d_out.float() * (a > 0)
        dz = dzf.to(torch.bfloat16).contiguous()
        cin = cins[name]
        grads[name + ".b"] = dzf.sum((0, 1, 2, 3))
        dw = TC.conv3x3x3_wgrad(dz, x)  # [Cout, 27, Cin']
        grads[name + ".w"] = dw[:, :, :cin].reshape(dw.shape[0], 3, 3, 3, cin).permute(0, 4, 1, 2, 3).contiguous()
        return TC.conv3x3x3_dgrad(dz, q[name][0], out_bf16=False) if need_dx else None

    d = layer("d1b", dh)
    d = layer("d1a", d)
    d_up1, d_e1 = d[..., :128], d[..., 128:]
    d = layer("d2b", _downsum(d_up1))
    d = layer("d2a", d)
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


def _pow2(v):
    return v > 0 and v & (v - 1) == 0


def tile_shape(D, H, W):
    """(D', H', W') >= (D, H, W), each a multiple of 4 (two poolings), that the
    3x3x3 kernel tiles at all three levels: at each level the width is a
    multiple of 128 or a power of two; below 128 the height is a multiple of
    128 / width, or (planes smaller than 128 voxels) both are powers of two and
    the depth a multiple of 128 / (height x width).  Chosen axis by axis,
    width first."""
    def w_ok(w):
        return w % 4 == 0 and all((w >> l) % 128 == 0 or _pow2(w >> l) for l in range(3))

    def h_ok(h, w):
        if h % 4:
            return False
        for l in range(3):
            hl, wl = h >> l, w >> l
            if wl < 128 and (hl % (128 // wl) if hl * wl >= 128 else not _pow2(hl)):
                return False
        return True

    def d_ok(d, h, w):
        return d % 4 == 0 and all((h >> l) * (w >> l) >= 128 or (d >> l) % (128 // ((h >> l) * (w >> l))) == 0
                                  for l in range(3))

    Wp = W
    while not w_ok(Wp):
        Wp += 1
    Hp = H
    while not h_ok(Hp, Wp):
        Hp += 1
    Dp = D
    while not d_ok(Dp, Hp, Wp):
        Dp += 1
    return Dp, Hp, Wp


def train(p, patches, steps, batch=8, lr=2e-3, sigma_range=(0.02, 3.0), seed=0, log_every=0, backend="torch"):
    """Adam on E || x0-hat(x0 + sigma eps, sigma) - x0 ||^2, sigma log-uniform,
    over FP32 volume patches [N, S, S, S] on the device; backend "torch"
    (autograd FP32) or "tc" (tcgen05 forward and backward, FP32 master weights)."""
    keys = list(p.keys())
    if backend == "torch":
        for v in p.values():
            v.requires_grad_(True)
    opt = torch.optim.Adam([p[k] for k in keys], lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    g = torch.Generator(device=patches.device).manual_seed(seed)
    lo, hi = math.log(sigma_range[0]), math.log(sigma_range[1])
    hist = []
    for k in range(steps):
        idx = torch.randint(0, patches.shape[0], (batch,), device=patches.device, generator=g)
        x0 = patches[idx]
        sig = torch.exp(lo + (hi - lo) * torch.rand(batch, device=patches.device, generator=g))
        y = (x0 + sig.view(-1, 1, 1, 1) * torch.randn(x0.shape, device=patches.device, generator=g)).contiguous()
        if backend == "torch":
            loss = F.mse_loss(forward_torch(p, y, sig), x0)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            val = float(loss.detach()) if log_every and k % log_every == 0 else None
        else:
            q = pack(p)
            xh, saved = forward_tc_train(q, y, sig)
            r = xh - x0
            grads = backward_tc(q, saved, (2.0 / r.numel()) * r)
            for key in keys:
                p[key].grad = grads[key].view_as(p[key])
            val = float((r * r).mean()) if log_every and k % log_every == 0 else None
        opt.step()
        sched.step()
        if val is not None:
            hist.append(val)
    for key in keys:
        p[key].requires_grad_(False)
        p[key].grad = None
    return hist


class UNet3DDenoiser:
    """x0-hat predictor for 3D models: (x_t [n, nz, ny, nx], abar_t) -> x0-hat
    in normalised units, on the tcgen05 kernels over the volume edge-padded to
    a tileable shape."""

    def __init__(self, params):
        self.q = pack(params)

    def __call__(self, x_t, abar_t):
        n, D, H, W = x_t.shape
        sig = torch.full((n,), math.sqrt((1.0 - abar_t) / abar_t), device=x_t.device)
        Dp, Hp, Wp = tile_shape(D, H, W)
        return _forward_tc(self.q, x_t, D, H, W, Dp, Hp, Wp, 1.0 / math.sqrt(abar_t), sig)
