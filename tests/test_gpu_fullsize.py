"""Full-size parity in the configuration the benchmark times: the thrust-belt
grid (801 x 187 at 25 m, 20-cell sponge, 2000 steps, 100 sources, 400
receivers) with 16 posterior samples x 5 supergathers of 20 +-1-encoded
shots in one call.  The FP64 oracle recomputes sampled outputs: the misfit
and gradient of one sample (five supergather solves) and the records of one
wavefield of another sample."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_thrust_belt_batch_sampled_parity():
    import torch
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    w = synth.thrust2d()
    g = O.Grid.from_workload(w)
    vel = synth.sample_models(w, w.nsamp, seed=100)
    d_obs = synth.random_records(w, 200)
    encs = [P.encode(1234 + s, 7, w.ns) for s in range(w.nsamp)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    B = w.nsamp * len(w.sg_sizes)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, B, 0)
    v_d = torch.tensor(vel).cuda()
    mis, grad = ctx.gradient(v_d, perm, wt, w.sg_sizes, torch.tensor(d_obs).cuda(), 1.0)
    rec = ctx.forward(v_d, perm, wt, w.sg_sizes)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    s = 5  # sampled posterior sample
    phi, gref = O.gradient(g, vel[s], w.src, w.rec, d_obs, perm[s], wt[s], w.sg_sizes, 1.0)
    e_phi = abs(mis[s].item() - phi) / abs(phi)
    e_g = rel(grad[s].cpu().numpy(), gref)
    assert e_phi < 1e-5 and e_g < 1e-4, (e_phi, e_g)
    s2, j2 = 11, 3  # sampled wavefield of another sample
    ref = O.encoded_forward(g, vel[s2], w.src, w.rec, perm[s2], wt[s2], w.sg_sizes)[j2]
    e_d = rel(rec[s2, j2].cpu().numpy(), ref)
    assert e_d < 1e-5, e_d


def _batch(P, w, enc_seed):
    encs = [P.encode(enc_seed + s, 7, w.ns) for s in range(w.nsamp)]
    return np.stack([e[0] for e in encs]), np.stack([e[1] for e in encs])


def _sampled_gradient_and_records(w, s, s2, j2):
    """One batched gradient and one batched forward call of the whole
    workload; the oracle recomputes sample s's misfit and gradient (all its
    supergathers) and the records of supergather j2 of sample s2."""
    import torch
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    g = O.Grid.from_workload(w)
    vel = synth.sample_models(w, w.nsamp, seed=100)
    d_obs = synth.random_records(w, 200)
    perm, wt = _batch(P, w, 4321)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, w.nsamp * len(w.sg_sizes), 0)
    try:
        v_d = torch.tensor(vel).cuda()
        mis, grad = ctx.gradient(v_d, perm, wt, w.sg_sizes, torch.tensor(d_obs).cuda(), 1.0)
        rec = ctx.forward(v_d, perm, wt, w.sg_sizes)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
        plan = ctx.plan_info()
        mis_s, grad_s, rec_s = mis[s].item(), grad[s].cpu().numpy(), rec[s2, j2].cpu().numpy()
    finally:
        ctx.close()
    phi, gref = O.gradient(g, vel[s], w.src, w.rec, d_obs, perm[s], wt[s], w.sg_sizes, 1.0)
    e_phi = abs(mis_s - phi) / abs(phi)
    e_g = rel(grad_s, gref)
    ref = O.encoded_forward(g, vel[s2], w.src, w.rec, perm[s2], wt[s2], w.sg_sizes)[j2]
    e_d = rel(rec_s, ref)
    return e_phi, e_g, e_d, plan


def test_salt_batch_sampled_parity():
    """Salt workload at full size: 676 x 210 at 20 m, 2000 steps, 130 sources
    in 5 supergathers of 26, a receiver on every node, 16 samples."""
    e_phi, e_g, e_d, _ = _sampled_gradient_and_records(synth.salt2d(), 9, 2, 4)
    assert e_phi < 1e-5 and e_g < 1e-4 and e_d < 1e-5, (e_phi, e_g, e_d)


def test_arid_uneven_batch_sampled_parity():
    """Near-surface workload at full size: 1001 x 201 at 10 m, 4000 steps,
    200 sources on a rough surface in uneven supergathers of 10 to 40 shots,
    8 samples (64 wavefields).  The sampled gradient covers all eight
    supergathers of one sample; the records are those of a 40-shot one."""
    w = synth.arid2d()
    e_phi, e_g, e_d, plan = _sampled_gradient_and_records(w, 6, 3, 4)
    assert e_phi < 1e-5 and e_g < 1e-4 and e_d < 1e-5, (e_phi, e_g, e_d, plan)


def test_arid_32_samples_uneven_batch_sampled_parity():
    """The top of the near-surface workload's batch range: 32 posterior
    samples x 8 uneven supergathers of 10 to 40 shots (256 wavefields of
    250,881 padded points, 4000 steps) in one call, which the library
    processes with checkpointing and, where that is cheaper, in chunks of
    samples.  The oracle recomputes one late sample's misfit and gradient
    (all eight supergathers) and the records of a 40-shot supergather of
    another."""
    w = synth.arid2d(nsamp=32)
    e_phi, e_g, e_d, plan = _sampled_gradient_and_records(w, 27, 13, 3)
    assert e_phi < 1e-5 and e_g < 1e-4 and e_d < 1e-5, (e_phi, e_g, e_d, plan)


def test_layered3d_batch_sampled_records_and_directional_derivative():
    """3D layered workload at full size: 256 x 256 x 128 at 20 m, 1500 steps,
    64 sources in 4 supergathers of 16, 4096 receivers, 8 samples (32
    wavefields of 14.7 M padded points) in one call.

    - Records: the oracle recomputes the first 750 steps of one wavefield.
      Records up to step n depend on the first n steps only, so a shorter
      oracle run gives an exact sample of the full one.
    - Gradient: the full 3D gradient of one sample is beyond the oracle's
      reach (its stored-wavefield adjoint would hold 177 GB), so the test
      checks a property that holds at any size: samples 1 and 2 are sample
      0 moved by +eps and -eps along a smooth direction dv, all with sample
      0's encoding, and the central difference of their misfits must match
      <grad_0, dv> (Sec. 2.1's gradient is the exact gradient of the
      discrete misfit)."""
    import torch
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    w = synth.layered3d()
    nsg = len(w.sg_sizes)
    vel = synth.sample_models(w, w.nsamp, seed=100)
    dv = synth.models.random_smooth_model(w.shape, 77, -1.0, 1.0, 4.0).astype(np.float64)
    eps = 5.0                                    # m/s at the peak of dv
    # the library refuses velocities above the grid's bound (FWI_ERR_CFL), so
    # the perturbed copies must stay inside [vmin, vmax]
    vel[0] = np.clip(vel[0], w.vmin + 2 * eps, w.vmax - 2 * eps)
    vel[1] = vel[0] + eps * dv
    vel[2] = vel[0] - eps * dv
    perm, wt = _batch(P, w, 999)
    perm[1:3], wt[1:3] = perm[0], wt[0]
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, w.nsamp * nsg, 0)
    try:
        v_d = torch.tensor(vel).cuda()
        rec = ctx.forward(v_d, perm, wt, w.sg_sizes)
        # observed data at a tenth of the predicted records' RMS, so the
        # misfit is shaped by the model rather than by the data
        d_rand = synth.random_records(w, 200)
        scale = 0.1 * float(rec.double().pow(2).mean().sqrt()) / float(np.sqrt(np.mean(d_rand.astype(np.float64) ** 2)))
        d_obs = torch.tensor(d_rand * np.float32(scale)).cuda()
        mis, grad = ctx.gradient(v_d, perm, wt, w.sg_sizes, d_obs, 1.0)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
        s2, j2, nsteps = 5, 2, 750
        rec_s = rec[s2, j2, :nsteps].cpu().numpy()
        mis = mis.cpu().numpy()
        # <grad_0, v_1 - v_2> with the FP32-rounded step
        dd = float((grad[0].double() * (v_d[1].double() - v_d[2].double())).sum())
    finally:
        ctx.close()
    assert abs((mis[1] - mis[2]) - dd) < 1e-2 * abs(dd), (mis[1] - mis[2], dd, mis[:3])
    wshort = synth.layered3d(nt=nsteps)
    ref = O.encoded_forward(O.Grid.from_workload(wshort), vel[s2], w.src, w.rec, perm[s2], wt[s2],
                            w.sg_sizes)[j2]
    e_d = rel(rec_s, ref)
    assert e_d < 1e-5, e_d


def test_layered3d_full_grid_gradient_matches_oracle_elementwise():
    # The whole 256 x 256 x 128 grid (296 x 296 x 168 padded) with its full
    # acquisition (64 sources as 4 supergathers of 16, 64 x 64 receivers),
    # one posterior sample, on the first 100 steps, so that the oracle's
    # stored FP64 snapshots fit in host memory (100 x 14.7 M x 8 B per
    # supergather).  Every tile of the grid takes part: receivers cover the
    # whole surface, so the adjoint source and the gradient reach every x-y
    # tile.  Gradient relative L2 <= 1e-4 and misfit <= 1e-5 against the
    # oracle, element by element over the whole grid.
    import torch
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    w = synth.layered3d(nt=100)
    g = O.Grid.from_workload(w)
    vel = synth.sample_models(w, 1, seed=101)
    d_obs = synth.random_records(w, 201)
    perm, wt = P.encode(4321, 3, w.ns)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, len(w.sg_sizes), 0)
    try:
        mis, grad = ctx.gradient(torch.tensor(vel).cuda(), perm, wt, w.sg_sizes, torch.tensor(d_obs).cuda(), 1.0)
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
        mis = mis.cpu().numpy()
        grad = grad.cpu().numpy()
    finally:
        ctx.close()
    phi, gref = O.gradient(g, vel[0], w.src, w.rec, d_obs, perm, wt, w.sg_sizes, 1.0)
    e_phi = abs(mis[0] - phi) / abs(phi)
    e_g = rel(grad[0], gref)
    # the gradient is not confined to a few tiles
    nz_tiles = (np.abs(gref).reshape(w.nz, 8, 32, 8, 32).max(axis=(0, 2, 4)) > 0).sum()
    assert nz_tiles == 64
    assert e_phi < 1e-5 and e_g < 1e-4, (e_phi, e_g)
