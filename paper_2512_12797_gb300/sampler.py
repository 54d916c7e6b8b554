"""Posterior samplers driven by the library's kernels.

encoded_diffusion_sampler -- the decoupled, encoded-shot sampler of Sec. 2.3:
    warm start at level t_start from the noised initial model (Sec. 2.2 and
    3.2), then for every level t: predict the clean model x0^ (Sec. 2.3 (i)),
    on guided levels run K clean-space Langevin steps with the unbiased
    encoded gradient (Sec. 2.3 (ii), supergathers redrawn every step,
    Sec. 3.2), and draw x_{t-1} from the DDPM posterior (Sec. 2.3 (iii)).
plain_langevin -- the baseline: unadjusted Langevin on the full-shot
    likelihood (every shot its own solve) plus a Gaussian smoothness prior.

Both use the same Langevin kernel and the same reading of the step size "in
physical units" (Sec. 2.3 (ii)): the gradient term is preconditioned per
element by the running root-mean-square of that element's gradient (the
diagonal preconditioner of preconditioned SGLD, Li et al. 2016, the Langevin
counterpart of the Adam refinement of Sec. 3.2), so each step moves an
element by about eta m/s; the independent noise has standard deviation nu
m/s.

The clean-model predictor is any callable (x_t, abar_t) -> x0^: the learned
network g_theta of Sec. 2.2 (unet.UNetDenoiser, unet3d.UNet3DDenoiser on the
tensor-core kernels) or, by default, the exact MMSE denoiser of a stationary
Gaussian prior on the normalised model (diagonal in Fourier space).

The encoded sampler can stop before a level and resume from the returned
state: every random draw after the initial one is counter-based (encodings
from (seed, step), Langevin noise from (seed, step), re-noise from (seed,
level)), so a resumed run is bit-identical to an uninterrupted one.

Cost is counted as eq. pde-count: one forward and one adjoint solve per
supergather per gradient evaluation.
"""
import math
import time

import numpy as np

from . import encode, langevin_step, renoise


def ddpm_schedule(T=1000, beta1=1e-4, betaT=0.02):
    """Linear beta schedule, cumulative alpha (Sec. 2.2; T = 1000, linear, Sec. 3.1)."""
    beta = np.linspace(beta1, betaT, T)
    return beta, np.cumprod(1.0 - beta)


def normalize(v, vmin, vmax):
    """Velocities to [-1, 1] (Sec. 2.2)."""
    return 2.0 * (v - vmin) / (vmax - vmin) - 1.0


def unnormalize(x, vmin, vmax):
    return vmin + 0.5 * (x + 1.0) * (vmax - vmin)


class GaussianPriorDenoiser:
    """x0^ = E[x0 | x_t] for a stationary Gaussian prior x0 ~ N(m, C) on the
    normalised model, C with spectrum amp^2 (1 + (k l)^2)^-2 (periodic
    approximation).  With y = x_t / sqrt(abar_t) = x0 + sigma e,
    sigma^2 = (1 - abar_t)/abar_t:  x0^ = m + F^-1[S / (S + sigma^2) F(y - m)]."""

    def __init__(self, mean, corr_cells=6.0, amp=1.0):
        import torch
        self.mean = mean
        shape = tuple(mean.shape)  # the model's axes: (nz, nx) or (nz, ny, nx)
        nd = len(shape)
        k2 = 0.0
        for a, n in enumerate(shape):
            f = torch.fft.rfftfreq(n, device=mean.device) if a == nd - 1 else torch.fft.fftfreq(n, device=mean.device)
            k = f * 2 * math.pi
            k2 = k2 + (k ** 2).view([-1 if b == a else 1 for b in range(nd)])
        # spectral density per Fourier mode, normalised so the pointwise variance is amp^2
        S = (1.0 + k2 * corr_cells ** 2) ** -2
        S = S / S.mean() * amp ** 2
        self.S = S
        self.dims = tuple(range(-len(shape), 0))

    def __call__(self, x_t, abar_t):
        import torch
        sig2 = (1.0 - abar_t) / abar_t
        y = x_t / math.sqrt(abar_t) - self.mean
        Y = torch.fft.rfftn(y, dim=self.dims)
        return self.mean + torch.fft.irfftn(Y * (self.S / (self.S + sig2)), s=y.shape[-len(self.dims):], dim=self.dims)


def _rmse(v, truth):
    return float(((v - truth) ** 2).mean().sqrt())


def _rms_normalise(grad):
    """Divide each sample's gradient by its root-mean-square value (in place)."""
    g = grad.reshape(grad.shape[0], -1)
    g.div_(g.pow(2).mean(dim=1).sqrt().clamp_min(1e-30)[:, None])


class RMSPreconditioner:
    """Diagonal preconditioner of preconditioned SGLD: g -> g / (sqrt(v) + eps),
    v the exponential moving average of g^2 per element (in place on g)."""

    def __init__(self, like, alpha=0.9, eps=1e-3):
        import torch
        self.v = torch.zeros_like(like)
        self.alpha, self.eps, self.n = alpha, eps, 0

    def state_dict(self):
        return {"v": self.v.clone(), "n": self.n}

    def load_state_dict(self, st):
        self.v.copy_(st["v"])
        self.n = int(st["n"])

    def __call__(self, g):
        self.n += 1
        self.v.mul_(self.alpha).addcmul_(g, g, value=1.0 - self.alpha)
        vhat = self.v / (1.0 - self.alpha ** self.n)
        g.div_(vhat.sqrt().add_(self.eps))


class AdamState:
    """Adam moments (Kingma & Ba 2015) for the deterministic refinement variant
    (A15): g -> m-hat / (sqrt(v-hat) + eps) in place, m and v the exponential
    moving averages of g and g^2 (beta1 0.9, beta2 0.999)."""

    def __init__(self, like, beta1=0.9, beta2=0.999, eps=1e-8):
        import torch
        self.m = torch.zeros_like(like)
        self.v = torch.zeros_like(like)
        self.b1, self.b2, self.eps, self.n = beta1, beta2, eps, 0

    def state_dict(self):
        return {"m": self.m.clone(), "v": self.v.clone(), "n": self.n}

    def load_state_dict(self, st):
        self.m.copy_(st["m"])
        self.v.copy_(st["v"])
        self.n = int(st["n"])

    def __call__(self, g):
        self.n += 1
        self.m.mul_(self.b1).add_(g, alpha=1.0 - self.b1)
        self.v.mul_(self.b2).addcmul_(g, g, value=1.0 - self.b2)
        mhat = self.m / (1.0 - self.b1 ** self.n)
        vhat = self.v / (1.0 - self.b2 ** self.n)
        g.copy_(mhat / (vhat.sqrt() + self.eps))


def _sync(t):
    import torch
    if t.is_cuda:
        torch.cuda.synchronize(t.device)


def plain_langevin(ctx, v0, d_obs, truth, steps, eta, nu, vmin, vmax, sigma, prior_lam=0.0, prior_mu=0.0,
                   zref=None, seed=0, record_every=1, sg_sizes=None):
    """Unadjusted Langevin on the full-shot likelihood (+ smoothness prior).

    Every gradient evaluation solves each shot separately (N_s supergathers
    of one shot, weight +1) -- or, with sg_sizes, uses the unbiased encoded
    gradient of supergathers of those sizes, redrawn every step (Sec. 2.1,
    3.2).  The RMS-normalised data gradient is combined with the gradient of
    the smoothness prior lam/2 |grad(z - zref)|^2 + mu/2 |z - zref|^2.
    Returns dict(rmse=[...], solves=[...], seconds, samples).
    """
    import torch
    z = v0.clone()
    ns = ctx.ns
    nsamp = z.shape[0]
    encoded = sg_sizes is not None
    if not encoded:
        perm = np.arange(ns, dtype=np.int32)
        w = np.ones(ns, np.int8)
        sg = [1] * ns
    else:
        sg = list(sg_sizes)
    hist_r, hist_s = [_rmse(z.mean(0), truth)], [0]
    zref = v0.mean(0) if zref is None else zref
    grad = torch.empty_like(z)
    precond = RMSPreconditioner(z)
    _sync(z)
    t0 = time.perf_counter()
    solves = 0
    for k in range(steps):
        if encoded:
            encs = [encode(seed * 7919 + i, k, ns) for i in range(nsamp)]
            perm = np.stack([e[0] for e in encs])
            w = np.stack([e[1] for e in encs])
        ctx.gradient(z, perm, w, sg, d_obs, sigma, scale=0.0 if encoded else 1.0, grad=grad)
        _rms_normalise(grad)
        if prior_lam > 0 or prior_mu > 0:
            ctx.smooth_prior_grad(z, zref.contiguous(), prior_lam, prior_mu, grad)
        precond(grad)
        langevin_step(z, grad, eta, nu, vmin, vmax, seed, k)
        solves += 2 * len(sg) * nsamp
        if (k + 1) % record_every == 0:
            hist_r.append(_rmse(z.mean(0), truth))
            hist_s.append(solves)
    _sync(z)
    return {"rmse": hist_r, "solves": hist_s, "seconds": time.perf_counter() - t0, "samples": z}


def encoded_diffusion_sampler(ctx, v_init, d_obs, truth, nsamp, sg_sizes, t_start, stride, K, eta, nu, vmin, vmax,
                              sigma, denoiser=None, seed=0, renoise_on=True, refine="langevin", state=None,
                              stop_at=None):
    """Decoupled encoded-shot diffusion sampler (Sec. 2.3, Algorithm table).

    refine: "langevin" -- K Langevin steps per guided level (Sec. 2.3 (ii));
            "adam"     -- K deterministic Adam steps on the same encoded
                          likelihood instead (the deterministic refinement of
                          Sec. 3.2, A15), no injected noise.  The two differ only
                          there, which is the stochastic-vs-deterministic
                          refinement ablation (E10).

    v_init: [nz, nx] initial model (m/s).  Starts from level t_start with
    x_t = sqrt(abar) x_init + sqrt(1 - abar) eps; guided levels are every
    `stride`-th level, each with K Langevin steps on the encoded likelihood
    with the given supergather sizes.  Returns dict(rmse, solves, seconds,
    samples) with the posterior-mean RMSE after every guided level.

    Checkpoint and resume: with stop_at = t the run stops before level t and
    returns samples=None and a "state" (plain tensors and numbers, e.g. for
    torch.save); passing it back as state= with the same other arguments
    continues at level t, bit-identically to an uninterrupted run.
    """
    import torch
    beta, abar = ddpm_schedule()
    dev = v_init.device
    x_init = normalize(v_init, vmin, vmax)
    if denoiser is None:
        denoiser = GaussianPriorDenoiser(x_init)
    if refine not in ("langevin", "adam"):
        raise ValueError("refine must be 'langevin' or 'adam'")
    run_key = [int(seed), int(nsamp), [int(v) for v in sg_sizes], int(t_start), int(stride), int(K), refine,
               bool(renoise_on)]
    shape = (nsamp,) + tuple(v_init.shape)
    if state is None:
        gen = torch.Generator(device=dev).manual_seed(seed)
        x_t = (math.sqrt(abar[t_start - 1]) * x_init[None] +
               math.sqrt(1 - abar[t_start - 1]) * torch.randn(shape, device=dev, generator=gen)).contiguous()
    else:
        if state["run"] != run_key:
            raise ValueError("state was saved by a run with other arguments: %s" % (state["run"],))
        x_t = state["x_t"].to(dev).clone().contiguous()
    grad = torch.empty_like(x_t)
    precond = RMSPreconditioner(x_t) if refine == "langevin" else AdamState(x_t)
    step_nu = nu if refine == "langevin" else 0.0
    if state is None:
        hist_r, hist_s = [_rmse(v_init, truth)], [0]
        solves, it, t_first = 0, 0, t_start
    else:
        precond.load_state_dict({k: (v.to(dev) if hasattr(v, "to") else v) for k, v in state["precond"].items()})
        hist_r, hist_s = list(state["rmse"]), list(state["solves"])
        solves, it, t_first = int(state["solves_total"]), int(state["it"]), int(state["t"])
    nsg = len(sg_sizes)
    _sync(x_t)
    t0 = time.perf_counter()
    z = None
    for t in range(t_first, 0, -1):
        if stop_at is not None and t == stop_at:
            _sync(x_t)
            st = {"run": run_key, "t": t, "x_t": x_t.clone(), "it": it, "solves_total": solves,
                  "rmse": list(hist_r), "solves": list(hist_s), "precond": precond.state_dict()}
            return {"rmse": hist_r, "solves": hist_s, "seconds": time.perf_counter() - t0, "samples": None,
                    "state": st}
        x0 = denoiser(x_t, abar[t - 1]).clamp(-1.0, 1.0)
        if t % stride == 0 or t == 1:
            z = unnormalize(x0, vmin, vmax).contiguous()
            for k in range(K):
                encs = [encode(seed * 7919 + s, it, ctx.ns) for s in range(nsamp)]
                perm = np.stack([e[0] for e in encs])
                w = np.stack([e[1] for e in encs])
                ctx.gradient(z, perm, w, sg_sizes, d_obs, sigma, grad=grad)
                if refine == "langevin":
                    _rms_normalise(grad)
                precond(grad)
                langevin_step(z, grad, eta, step_nu, vmin, vmax, seed + 1, it)
                solves += 2 * nsg * nsamp
                it += 1
            x0 = normalize(z, vmin, vmax).contiguous()
            hist_r.append(_rmse(z.mean(0), truth))
            hist_s.append(solves)
        if t > 1:
            if renoise_on:
                x_t = renoise(x_t.contiguous(), x0.contiguous(), abar[t - 1], abar[t - 2], beta[t - 1], seed + 2, t)
            else:
                x_t = (math.sqrt(abar[t - 2]) * x0).contiguous()
    _sync(x_t)
    return {"rmse": hist_r, "solves": hist_s, "seconds": time.perf_counter() - t0,
            "samples": unnormalize(x0, vmin, vmax)}
