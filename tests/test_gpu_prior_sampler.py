"""The learned prior inside the sampler (Sec. 2.2, 2.3 (i), 3.3).  On the salt
workload (676 x 210 at 20 m, 130 sources in 5 supergathers of 26, a
receiver on every node, 2000 steps, data from the forward on the seeded
truth plus 1 % noise), the encoded diffusion sampler runs the paper's
schedule for this case -- 50 guided levels (every 6th of the last 300) x 10
preconditioned Langevin steps -- once with the U-Net trained on the
library's kernels as its clean-model predictor and once with the Gaussian
smoothness prior's exact MMSE denoiser (the method without the learned
part), at equal PDE solves.  The learned prior must give the lower
posterior-mean model RMSE and data misfit; the posterior spread of each arm
is printed.

Only the batch is scaled down from the workload's 16 samples: 4 posterior
samples per arm.  The network is trained for 800 Adam steps on 8,192 seeded
salt-style 64 x 64 patches (synth.patches)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_learned_prior_lowers_posterior_rmse_and_misfit_on_salt():
    import torch
    import synth.patches as SP
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    from paper_2512_12797_gb300 import sampler as S, unet

    w = synth.salt2d()
    nsamp = 4
    truth = torch.tensor(synth.true_model(w)).cuda()
    vinit = torch.tensor(synth.initial_model(w)).cuda()
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, nsamp * w.ns, 0)
    ident = np.arange(w.ns, dtype=np.int32)
    ones = np.ones(w.ns, np.int8)
    d_clean = ctx.forward(truth[None].contiguous(), ident, ones, [1] * w.ns)[0]
    gen = torch.Generator(device="cuda").manual_seed(3)
    noise = 0.01 * float(d_clean.pow(2).mean().sqrt())
    d_obs = (d_clean + noise * torch.randn(d_clean.shape, device="cuda", generator=gen)).contiguous()

    patches = torch.tensor(SP.geology_patches(8192, 64, 21, styles=("salt",))).cuda()
    params = unet.init_params(0)
    hist = unet.train(params, patches, steps=800, batch=64, lr=2e-3, seed=1, log_every=100)
    assert hist[-1] < 0.1 * hist[0]

    def nrms(samples):
        d = ctx.forward(samples.contiguous(), ident, ones, [1] * w.ns)
        return float((d - d_obs[None]).pow(2).sum().sqrt() / d_obs[None].expand_as(d).pow(2).sum().sqrt())

    kw = dict(nsamp=nsamp, sg_sizes=w.sg_sizes, t_start=300, stride=6, K=10, eta=10.0, vmin=w.vmin,
              vmax=w.vmax, sigma=noise, seed=5)
    runs = {"unet": S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, denoiser=unet.UNetDenoiser(params), **kw),
            "gaussian": S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, **kw)}
    out = {}
    for name, r in runs.items():
        s = r["samples"]
        out[name] = (r["rmse"][-1], float(s.std(0).mean()), nrms(s), r["solves"][-1])
        print("%-8s posterior-mean RMSE %.1f m/s, spread %.1f m/s, data NRMS %.3f, %d PDE solves"
              % ((name,) + out[name]))
    assert out["unet"][3] == out["gaussian"][3] == 2 * len(w.sg_sizes) * nsamp * 10 * (300 // 6 + 1)
    assert out["unet"][0] < 0.8 * out["gaussian"][0]
    assert out["unet"][0] < runs["unet"]["rmse"][0]
    assert out["unet"][2] < out["gaussian"][2]
    ctx.close()


def test_learned_3d_prior_lowers_posterior_rmse_on_layered3d():
    """The 3D workload (256 x 256 x 128 at 20 m, 64 sources in 4 supergathers
    of 16, 64 x 64 receivers, 1500 steps; data from the forward on the seeded
    truth plus 1 % noise) with the 3D U-Net trained on the library's kernels
    (1,500 Adam steps on 512 seeded 32^3 layered-and-faulted patches) against
    the Gaussian MMSE denoiser, at equal PDE solves.  Scaled down from the
    workload's 8 samples x 300 levels in batch and levels only: 2 posterior
    samples, 10 guided levels (every 6th of the last 60, and level 1) x 2
    preconditioned Langevin steps."""
    import torch
    import synth.patches as SP
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    from paper_2512_12797_gb300 import sampler as S, unet3d

    w = synth.layered3d()
    nsamp = 2
    truth = torch.tensor(synth.true_model(w)).cuda()
    vinit = torch.tensor(synth.initial_model(w)).cuda()
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, w.ns, 120 << 30)
    ident = np.arange(w.ns, dtype=np.int32)
    d_clean = ctx.forward(truth[None].contiguous(), ident, np.ones(w.ns, np.int8), [1] * w.ns)[0]
    gen = torch.Generator(device="cuda").manual_seed(3)
    noise = 0.01 * float(d_clean.pow(2).mean().sqrt())
    d_obs = (d_clean + noise * torch.randn(d_clean.shape, device="cuda", generator=gen)).contiguous()
    del d_clean

    patches = torch.tensor(SP.volume_patches(512, 32, 21)).cuda()
    params = unet3d.init_params(0)
    unet3d.train(params, patches, steps=1500, batch=8, lr=2e-3, seed=3, backend="tc")
    kw = dict(nsamp=nsamp, sg_sizes=w.sg_sizes, t_start=60, stride=6, K=2, eta=10.0, vmin=w.vmin, vmax=w.vmax,
              sigma=noise, seed=5)
    out = {}
    for name, den in (("unet3d", unet3d.UNet3DDenoiser(params)), ("gaussian", None)):
        r = S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, denoiser=den, **kw)
        out[name] = (r["rmse"][-1], float(r["samples"].std(0).mean()), r["solves"][-1])
        print("%-8s posterior-mean RMSE %.1f m/s, spread %.1f m/s, %d PDE solves" % ((name,) + out[name]))
    assert out["unet3d"][2] == out["gaussian"][2] == 2 * len(w.sg_sizes) * nsamp * 2 * (60 // 6 + 1)
    assert out["unet3d"][0] < 0.7 * out["gaussian"][0]
    assert out["unet3d"][1] < out["gaussian"][1]
    ctx.close()
