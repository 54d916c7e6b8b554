"""Posterior samplers driven by the library's kernels.

encoded_diffusion_sampler -- the decoupled, encoded-shot sampler of Sec. 2.3:
    warm start at level t_start from the noised initial model (Sec. 2.2 and
    3.2), then for every level t: predict the clean model x0^ (Sec. 2.3 (i)),
    on guided levels run K clean-space Langevin steps with the unbiased
    encoded gradient (Sec. 2.3 (ii), supergathers redrawn every step,
    Sec. 3.2), and draw x_{t-1} from the DDPM posterior (Sec. 2.3 (iii)).
plain_langevin -- the baseline: unadjusted Langevin on the full-shot
    likelihood (every shot its own solve) plus a Gaussian smoothness prior.

Both use the same refinement kernel (langevin_step_precond) with the
paper's requirement that the noise be matched to any preconditioning
(Sec. 5): the drift is preconditioned per element by the running
root-mean-square of that element's gradient (RMSprop second moment, the
diagonal preconditioner G of preconditioned SGLD, Li et al. 2016), and the
injected noise is nu sqrt(G) xi with nu = sqrt(2 eta) by default, so the
chain targets the tempered posterior of Sec. 2.3 up to the step's O(eta)
bias.  eta is a step in m/s ("physical units", Sec. 2.3 (ii)): a step
moves a well-informed element by about eta.  The preconditioner's damping
eps is relative to each sample's gradient scale.  A different nu is the
paper's independent noise scale (Sec. 2.3, closing paragraph).  The
deterministic variant (refine="adam") runs Adam through the same kernel
with nu = 0.  Every update runs in the library: no PyTorch arithmetic sits
between the gradient and the step.

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

from . import encode, renoise


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


class Moments:
    """Moment buffers of the refinement kernel: the second moment v (and, for
    Adam, the first moment m) per element, plus the step count k of the bias
    correction.  Plain tensors, so a sampler state can be saved and resumed."""

    def __init__(self, like, adam=False):
        import torch
        self.v = torch.zeros_like(like)
        self.m = torch.zeros_like(like) if adam else None
        self.k = 0

    def state_dict(self):
        st = {"v": self.v.clone(), "k": self.k}
        if self.m is not None:
            st["m"] = self.m.clone()
        return st

    def load_state_dict(self, st):
        self.v.copy_(st["v"])
        if self.m is not None:
            self.m.copy_(st["m"])
        self.k = int(st["k"])


def refine_step(ctx, z, grad, mom, eta, nu, vmin, vmax, seed, counter, eps=0.1, adam=False):
    """One refinement step in place on z (langevin_step_precond): the
    preconditioned Langevin step with matched noise, or with adam=True an
    Adam step (beta1 0.9, beta2 0.999, no noise)."""
    mom.k += 1
    if adam:
        return ctx.langevin_precond(z, grad, mom.v, mom.k, eta, 0.0, vmin, vmax, seed, counter, m=mom.m, alpha=0.999,
                                    beta1=0.9, eps=eps)
    return ctx.langevin_precond(z, grad, mom.v, mom.k, eta, nu, vmin, vmax, seed, counter, alpha=0.9, eps=eps)


def _sync(t):
    import torch
    if t.is_cuda:
        torch.cuda.synchronize(t.device)


def plain_langevin(ctx, v0, d_obs, truth, steps, eta, vmin, vmax, sigma, nu=None, prior_lam=0.0, prior_mu=0.0,
                   zref=None, seed=0, record_every=1, sg_sizes=None, eps=0.1, rmse_target=None):
    """Preconditioned Langevin on the full-shot likelihood (+ smoothness prior).

    Every gradient evaluation solves each shot separately (N_s supergathers
    of one shot, weight +1) -- or, with sg_sizes, uses the unbiased encoded
    gradient of supergathers of those sizes, redrawn every step (Sec. 2.1,
    3.2).  The data gradient plus the gradient of the smoothness prior
    lam/2 |grad(z - zref)|^2 + mu/2 |z - zref|^2 drives the preconditioned
    Langevin step (nu None: sqrt(2 eta), the posterior-targeting noise).
    With rmse_target the run stops at the first recorded posterior-mean RMSE
    at or below it.  Returns dict(rmse=[...], solves=[...], seconds, samples,
    reached: solves and seconds when the target was first met, else None).
    """
    import torch
    nu = math.sqrt(2.0 * eta) if nu is None else nu
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
    zref = (v0.mean(0) if zref is None else zref).contiguous()
    grad = torch.empty_like(z)
    mom = Moments(z)
    _sync(z)
    t0 = time.perf_counter()
    solves = 0
    reached = None
    for k in range(steps):
        if encoded:
            encs = [encode(seed * 7919 + i, k, ns) for i in range(nsamp)]
            perm = np.stack([e[0] for e in encs])
            w = np.stack([e[1] for e in encs])
        ctx.gradient(z, perm, w, sg, d_obs, sigma, scale=0.0 if encoded else 1.0, grad=grad)
        if prior_lam > 0 or prior_mu > 0:
            ctx.smooth_prior_grad(z, zref, prior_lam, prior_mu, grad)
        refine_step(ctx, z, grad, mom, eta, nu, vmin, vmax, seed, k, eps=eps)
        solves += 2 * len(sg) * nsamp
        if (k + 1) % record_every == 0:
            hist_r.append(_rmse(z.mean(0), truth))
            hist_s.append(solves)
            if rmse_target is not None and hist_r[-1] <= rmse_target:
                _sync(z)
                reached = {"solves": solves, "seconds": time.perf_counter() - t0, "steps": k + 1}
                break
    _sync(z)
    return {"rmse": hist_r, "solves": hist_s, "seconds": time.perf_counter() - t0, "samples": z,
            "reached": reached}


def encoded_diffusion_sampler(ctx, v_init, d_obs, truth, nsamp, sg_sizes, t_start, stride, K, eta, vmin, vmax,
                              sigma, nu=None, denoiser=None, seed=0, renoise_on=True, refine="langevin", state=None,
                              stop_at=None, eps=0.1):
    """Decoupled encoded-shot diffusion sampler (Sec. 2.3, Algorithm table).

    refine: "langevin" -- K preconditioned Langevin steps with matched noise
                          per guided level (Sec. 2.3 (ii), Sec. 5; nu None:
                          sqrt(2 eta));
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
               bool(renoise_on), float(eta), None if nu is None else float(nu), float(eps)]
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
    nu = math.sqrt(2.0 * eta) if nu is None else nu
    precond = Moments(x_t, adam=(refine == "adam"))
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
                refine_step(ctx, z, grad, precond, eta, nu, vmin, vmax, seed + 1, it, eps=eps,
                            adam=(refine == "adam"))
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
