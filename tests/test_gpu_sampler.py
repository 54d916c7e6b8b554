"""Sampler behaviour on the small 2D case (8 shots, 1 s of data, 1 % noise)
and at equal model RMSE on the thrust-belt workload.

Cost (Sec. 2.4, eq. pde-count): encoded supergathers cut PDE solves per
refinement step by about the supergather size.  Langevin refinement with the
unbiased encoded gradient (one supergather of all 8 shots, redrawn every
step: 2 solves per step and sample) is given half the solve budget of the
full-shot Langevin baseline (16 solves per step and sample) and must reach
at least the same posterior-mean model RMSE against the seeded truth.  On
the thrust-belt geometry (100 shots in 5 supergathers of 20) the encoded
chain must reach the full-shot chain's RMSE with fewer solves and in less
time, i.e. at more posterior samples per hour.

Both chains take the preconditioned Langevin step with noise matched to the
preconditioner (nu = sqrt(2 eta), Sec. 5).

Calibration (Sec. 3.5 ablation): the decoupled diffusion sampler with DDPM
re-noising keeps a larger posterior spread than the same loop with the
noise removed.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _setup(nsamp):
    import torch
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    w = synth.small2d()
    truth_np = synth.true_model(w)
    vinit_np = synth.initial_model(w, truth_np)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, nsamp * w.ns, 1 << 31)
    truth = torch.tensor(truth_np).cuda()
    vinit = torch.tensor(vinit_np).cuda()
    ident = np.arange(w.ns, dtype=np.int32)
    d_clean = ctx.forward(truth[None].contiguous(), ident, np.ones(w.ns, np.int8), [1] * w.ns)[0]
    gen = torch.Generator(device="cuda").manual_seed(3)
    noise = 0.01 * float(d_clean.pow(2).mean().sqrt())
    d_obs = (d_clean + noise * torch.randn(d_clean.shape, device="cuda", generator=gen)).contiguous()
    return w, ctx, truth, vinit, d_obs, noise


def test_encoded_langevin_matches_full_shot_with_half_the_solves():
    from paper_2512_12797_gb300 import sampler as S
    nsamp = 4
    w, ctx, truth, vinit, d_obs, noise = _setup(nsamp)
    v0 = vinit[None].repeat(nsamp, 1, 1).contiguous()
    kw = dict(eta=10.0, vmin=w.vmin, vmax=w.vmax, sigma=noise, prior_lam=10.0, seed=5)
    plain = S.plain_langevin(ctx, v0, d_obs, truth, steps=40, **kw)
    enc = S.plain_langevin(ctx, v0, d_obs, truth, steps=160, sg_sizes=[w.ns], **kw)
    print("full-shot rmse %.1f -> %.1f m/s, %d solves, %.2f s" % (plain["rmse"][0], plain["rmse"][-1],
                                                                   plain["solves"][-1], plain["seconds"]))
    print("encoded   rmse %.1f -> %.1f m/s, %d solves, %.2f s" % (enc["rmse"][0], enc["rmse"][-1],
                                                                   enc["solves"][-1], enc["seconds"]))
    assert plain["rmse"][-1] < plain["rmse"][0]
    assert enc["solves"][-1] <= plain["solves"][-1] // 2
    assert enc["rmse"][-1] <= plain["rmse"][-1]


def test_diffusion_sampler_renoise_keeps_posterior_spread():
    import torch
    from paper_2512_12797_gb300 import sampler as S
    nsamp = 6
    w, ctx, truth, vinit, d_obs, noise = _setup(nsamp)
    kw = dict(nsamp=nsamp, sg_sizes=[w.ns], t_start=60, stride=2, K=1, eta=10.0, vmin=w.vmin,
              vmax=w.vmax, sigma=noise, seed=9)
    on = S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, **kw)
    off = S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, renoise_on=False, **kw)
    s_on = float(on["samples"].std(dim=0).mean())
    s_off = float(off["samples"].std(dim=0).mean())
    print("posterior spread: renoise %.2f m/s, zero-variance %.2f m/s" % (s_on, s_off))
    assert torch.isfinite(on["samples"]).all() and torch.isfinite(off["samples"]).all()
    assert on["solves"][-1] == off["solves"][-1] == 2 * nsamp * (60 // 2 + 1)  # every 2nd level and t = 1
    assert s_on > 1.5 * s_off


def test_deterministic_adam_refinement_ablation():
    # Stochastic vs deterministic refinement (E10): the same schedule and
    # encodings with the K Langevin steps replaced by K Adam steps (A15, no
    # injected noise).  Both cost the same PDE solves.  On this case the
    # posterior spread is set by the encodings, which are redrawn at every step
    # (the encoded gradient is itself random), and by re-noising, not by the
    # refinement's own noise: the two spreads agree to within a factor of 2
    # with and without re-noising.  The numbers are printed for the record.
    import torch
    from paper_2512_12797_gb300 import sampler as S
    nsamp = 6
    w, ctx, truth, vinit, d_obs, noise = _setup(nsamp)
    for renoise_on in (True, False):
        kw = dict(nsamp=nsamp, sg_sizes=[w.ns], t_start=60, stride=2, K=2, eta=10.0, vmin=w.vmin,
                  vmax=w.vmax, sigma=noise, seed=11, renoise_on=renoise_on)
        lang = S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, refine="langevin", **kw)
        adam = S.encoded_diffusion_sampler(ctx, vinit, d_obs, truth, refine="adam", **kw)
        s_lang = float(lang["samples"].std(dim=0).mean())
        s_adam = float(adam["samples"].std(dim=0).mean())
        print("renoise %s: posterior spread Langevin %.2f m/s, Adam %.2f m/s; rmse %.1f / %.1f m/s"
              % (renoise_on, s_lang, s_adam, lang["rmse"][-1], adam["rmse"][-1]))
        assert torch.isfinite(adam["samples"]).all() and torch.isfinite(lang["samples"]).all()
        assert lang["solves"][-1] == adam["solves"][-1]
        assert 0.5 < s_adam / s_lang < 2.0


def test_encoded_reaches_full_shot_rmse_with_fewer_solves_and_more_samples_per_hour():
    # thrust-belt geometry and batch shape (100 shots, 5 supergathers of 20),
    # 4 posterior samples, the first 1000 steps; observed data from the
    # forward on the seeded truth plus 1 % noise.  The full-shot chain runs 8
    # steps; its final posterior-mean RMSE is the target the encoded chain
    # must reach (at most 20x the steps).
    import torch
    from paper_2512_12797_gb300 import build, sampler as S
    build.build()
    import paper_2512_12797_gb300 as P
    w = synth.thrust2d(nt=1000)
    nsamp = 4
    truth_np = synth.true_model(w)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, nsamp * w.ns, 0)
    truth = torch.tensor(truth_np).cuda()
    v0 = torch.tensor(synth.sample_models(w, nsamp, seed=7)).cuda()
    ident = np.arange(w.ns, dtype=np.int32)
    d_clean = ctx.forward(truth[None].contiguous(), ident, np.ones(w.ns, np.int8), [1] * w.ns)[0]
    gen = torch.Generator(device="cuda").manual_seed(4)
    noise = 0.01 * float(d_clean.pow(2).mean().sqrt())
    d_obs = (d_clean + noise * torch.randn(d_clean.shape, device="cuda", generator=gen)).contiguous()
    kw = dict(eta=15.0, vmin=w.vmin, vmax=w.vmax, sigma=noise, seed=3)
    full = S.plain_langevin(ctx, v0, d_obs, truth, steps=8, **kw)
    target = full["rmse"][-1]
    enc = S.plain_langevin(ctx, v0, d_obs, truth, steps=160, sg_sizes=w.sg_sizes, rmse_target=target, **kw)
    print("full shot: rmse %.1f -> %.1f m/s, %d solves, %.2f s" % (full["rmse"][0], target, full["solves"][-1],
                                                                   full["seconds"]))
    print("encoded  : reached %s" % (enc["reached"],))
    assert target < full["rmse"][0]
    assert enc["reached"] is not None
    assert enc["reached"]["solves"] < full["solves"][-1]
    sph_full = nsamp * 3600.0 / full["seconds"]
    sph_enc = nsamp * 3600.0 / enc["reached"]["seconds"]
    assert sph_enc > sph_full
