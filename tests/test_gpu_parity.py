"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 <= 1e-5 on forward records and <= 1e-4 on the
velocity gradient (FP32 device path vs FP64 oracle); +-1 encodings and
permutations bit-exact; Gaussian draws of the sampler updates within 1e-6
relative (FP64 on both sides, transcendental rounding only).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def P():
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    return P


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def make_ctx(P, w, max_wavefields, budget=1 << 30):
    return P.FWI(w.grid_dict(), w.src, w.rec, max_wavefields, budget)


def test_forward_small2d_single_shot(P, torch):
    w = synth.small2d()
    g = O.Grid.from_workload(w)
    v = synth.true_model(w)
    ctx = make_ctx(P, w, 1)
    ref = O.forward_shot(g, v, w.src[3:4], [1.0], w.rec)
    perm = np.array([3] + [i for i in range(w.ns) if i != 3], np.int32)
    d = ctx.forward(torch.tensor(v[None]).cuda(), perm, np.ones(w.ns, np.int8), [1])
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    e = rel(d[0, 0].cpu().numpy(), ref)
    assert e < FWD_TOL, e


def test_forward_small2d_encoded_supergather(P, torch):
    w = synth.small2d()
    g = O.Grid.from_workload(w)
    v = synth.true_model(w)
    perm, wt = P.encode(11, 4, w.ns)
    ref = O.encoded_forward(g, v, w.src, w.rec, perm, wt, [8])
    ctx = make_ctx(P, w, 1)
    d = ctx.forward(torch.tensor(v[None]).cuda(), perm, wt, [8])
    e = rel(d[0].cpu().numpy(), ref)
    assert e < FWD_TOL, e


def test_forward_linearity_on_device(P, torch):
    # Sec. 2.1: the encoded record equals the weighted sum of single-shot records.
    w = synth.small2d(nt=500)
    v = torch.tensor(synth.true_model(w)[None]).cuda()
    perm, wt = P.encode(5, 1, w.ns)
    ctx = make_ctx(P, w, w.ns)
    enc = ctx.forward(v, perm, wt, [w.ns])[0, 0].double()
    single = ctx.forward(v.repeat(1, 1, 1), perm, np.ones(w.ns, np.int8), [1] * w.ns)[0].double()
    s = sum(float(wt[perm[i]]) * single[i] for i in range(w.ns))
    # each FP32 record is within FWD_TOL of the exact one, so their difference is too
    e = rel(enc.cpu().numpy(), s.cpu().numpy())
    assert e < FWD_TOL, e


def test_gradient_small2d_matches_oracle(P, torch):
    w = synth.small2d()
    g = O.Grid.from_workload(w)
    truth = synth.true_model(w)
    v = synth.initial_model(w, truth)
    d_obs = np.stack([O.forward_shot(g, truth, w.src[i:i + 1], [1.0], w.rec) for i in range(w.ns)])
    perm, wt = P.encode(3, 0, w.ns)
    sigma = 1e-3
    phi_ref, g_ref = O.gradient(g, v, w.src, w.rec, d_obs, perm, wt, [8], sigma)
    ctx = make_ctx(P, w, 1)
    mis, grad = ctx.gradient(torch.tensor(v[None]).cuda(), perm, wt, [8],
                             torch.tensor(d_obs, dtype=torch.float32).cuda(), sigma)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    e_phi = abs(mis.item() - phi_ref) / abs(phi_ref)
    e_g = rel(grad[0].cpu().numpy(), g_ref)
    assert e_phi < 1e-5 and e_g < GRAD_TOL, (e_phi, e_g)


def test_gradient_batched_uneven_supergathers(P, torch):
    # several samples with their own encodings, uneven supergathers, ragged tiles
    w = synth.tiny2d(nz=45, nx=150, nt=250, ns=7, nr=20, nb=8)
    g = O.Grid.from_workload(w)
    nsamp, sg = 3, [4, 2, 1]
    rng = np.random.default_rng(0)
    vs = np.stack([synth.models.random_smooth_model(w.shape, 10 + s, 1500, 2500) for s in range(nsamp)])
    d_obs = synth.random_records(w, 5)
    encs = [P.encode(21, s, w.ns) for s in range(nsamp)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    ctx = make_ctx(P, w, nsamp * len(sg))
    mis, grad = ctx.gradient(torch.tensor(vs).cuda(), perm, wt, sg, torch.tensor(d_obs).cuda(), 0.5)
    torch.cuda.synchronize()
    for s in range(nsamp):
        phi_ref, g_ref = O.gradient(g, vs[s], w.src, w.rec, d_obs, perm[s], wt[s], sg, 0.5)
        e_phi = abs(mis[s].item() - phi_ref) / abs(phi_ref)
        e_g = rel(grad[s].cpu().numpy(), g_ref)
        assert e_phi < 1e-5 and e_g < GRAD_TOL, (s, e_phi, e_g)


def test_checkpointed_gradient_is_bit_exact(P, torch):
    # recomputing segments from checkpoints reproduces the stored-snapshot gradient bit for bit
    w = synth.tiny2d(nz=40, nx=70, nt=300, ns=4, nr=12, nb=6)
    v = torch.tensor(synth.models.random_smooth_model(w.shape, 3, 1500, 2500)[None]).cuda()
    d_obs = torch.tensor(synth.random_records(w, 2)).cuda()
    perm, wt = P.encode(1, 1, w.ns)
    big = make_ctx(P, w, 2, budget=1 << 30)
    m1, g1 = big.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    info_big = big.plan_info()
    # a budget of 80 slots of 2 wavefields forces segments + recompute
    field = (w.nz + 2 * w.nb + 8) * (((w.nx + 2 * w.nb + 8) + 31) // 32 * 32) * 4
    small = make_ctx(P, w, 2, budget=80 * 2 * field)
    m2, g2 = small.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    info_small = small.plan_info()
    torch.cuda.synchronize()
    assert info_big["recomputed_steps"] == 0
    assert info_small["recomputed_steps"] > 0 and info_small["segments"] > 1
    assert torch.equal(g1, g2) and torch.equal(m1, m2)


def test_langevin_matches_oracle(P, torch):
    n = 100003
    rng = np.random.default_rng(1)
    z = rng.uniform(1500, 3500, n).astype(np.float32)
    gr = rng.normal(0, 1, n).astype(np.float32)
    zt = torch.tensor(z).cuda()
    P.langevin_step(zt, torch.tensor(gr).cuda(), 30.0, 25.0, 1500.0, 3500.0, 77, 5)
    ref = O.langevin(z.astype(np.float64), gr.astype(np.float64), 30.0, 25.0, 1500.0, 3500.0, 77, 5)
    got = zt.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-6


def test_langevin_precond_matches_oracle(P, torch):
    # three consecutive preconditioned Langevin steps (noise matched to the
    # preconditioner) and three Adam steps on three samples whose gradients
    # differ in scale by 1e3, against the oracle; moments carried on both sides
    w = synth.tiny2d(nz=37, nx=53, nt=20)
    ctx = make_ctx(P, w, 3)
    rng = np.random.default_rng(4)
    shape = (3,) + w.shape
    z0 = rng.uniform(1600, 3400, shape).astype(np.float32)
    for use_m, nu in ((False, math.sqrt(2 * 20.0)), (True, 0.0)):
        zt = torch.tensor(z0).cuda()
        vt = torch.zeros_like(zt)
        mt = torch.zeros_like(zt) if use_m else None
        z, v, m = z0.astype(np.float64), np.zeros(shape), (np.zeros(shape) if use_m else None)
        for k in range(1, 4):
            g = (rng.normal(0, 1, shape) * np.array([1.0, 1e3, 1e-3])[:, None, None]).astype(np.float32)
            g[0, 5, 7] = 0.0
            ctx.langevin_precond(zt, torch.tensor(g).cuda(), vt, k, 20.0, nu, 1500.0, 3500.0, 31, 100 + k, m=mt,
                                 alpha=0.99, beta1=0.9, eps=1e-2)
            z, v, m = O.langevin_precond(z, g, v, m, 20.0, nu, 1500.0, 3500.0, 31, 100 + k, k=k, alpha=0.99,
                                         beta1=0.9, eps=1e-2)
            got = zt.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - z) / np.abs(z)) < 1e-6, (use_m, k)
            assert np.max(np.abs(vt.cpu().numpy() - v) / np.maximum(np.abs(v), 1e-30)) < 1e-6
            if use_m:
                assert np.max(np.abs(mt.cpu().numpy() - m)) < 1e-6 * np.max(np.abs(m))
    # invalid arguments are refused on the host
    zt = torch.tensor(z0).cuda()
    with pytest.raises(P.FwiError):
        ctx.langevin_precond(zt, zt.clone(), torch.zeros_like(zt), 3, 1.0, 1.0, 0.0, 1e4, 1, 1, alpha=1.0)
    with pytest.raises(ValueError, match="v"):
        ctx.langevin_precond(zt, zt.clone(), torch.zeros(3, 5, device="cuda"), 1, 1.0, 1.0, 0.0, 1e4, 1, 1)


def test_renoise_matches_oracle(P, torch):
    beta, abar = O.ddpm_schedule()
    t = 200
    n = 65536
    rng = np.random.default_rng(2)
    xt = rng.normal(0, 1, n).astype(np.float32)
    x0 = rng.uniform(-1, 1, n).astype(np.float32)
    out = P.renoise(torch.tensor(xt).cuda(), torch.tensor(x0).cuda(), abar[t - 1], abar[t - 2], beta[t - 1], 9, 3)
    ref = O.renoise(xt, x0, abar[t - 1], abar[t - 2], beta[t - 1], 9, 3)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))
    # first level: x_0 exactly
    out1 = P.renoise(torch.tensor(xt).cuda(), torch.tensor(x0).cuda(), abar[0], 1.0, beta[0], 9, 4)
    assert torch.equal(out1.cpu(), torch.tensor(x0))


def test_smooth_prior_matches_oracle(P, torch):
    w = synth.small2d()
    g = O.Grid.from_workload(w)
    rng = np.random.default_rng(4)
    z = (2500 + rng.normal(0, 50, (2,) + w.shape)).astype(np.float32)
    zr = synth.initial_model(w)
    ctx = make_ctx(P, w, 1)
    gr = torch.zeros(z.shape, device="cuda")
    ctx.smooth_prior_grad(torch.tensor(z).cuda(), torch.tensor(zr).cuda(), 2.0, 0.1, gr)
    for s in range(2):
        _, ref = O.smooth_prior(g, z[s], zr, 2.0, 0.1)
        assert rel(gr[s].cpu().numpy(), ref) < 1e-6


def test_nonfinite_misfit_sets_status(P, torch):
    w = synth.tiny2d(nt=50)
    ctx = make_ctx(P, w, 1)
    v = torch.tensor(synth.models.random_smooth_model(w.shape, 1, 1500, 2500)[None]).cuda()
    d_obs = torch.tensor(synth.random_records(w, 1)).cuda()
    d_obs[0, 10, 3] = float("nan")
    perm, wt = P.encode(0, 0, w.ns)
    ctx.gradient(v, perm, wt, [w.ns], d_obs, 1.0)
    assert ctx.device_status() == -5
    d_obs[0, 10, 3] = 0.0
    ctx.gradient(v, perm, wt, [w.ns], d_obs, 1.0)
    assert ctx.device_status() == 0


def test_velocity_above_stability_bound_sets_status(P, torch):
    w = synth.tiny2d(nt=20)
    ctx = make_ctx(P, w, 1)
    v = torch.full((1,) + w.shape, 2000.0, device="cuda")
    v[0, 5, 5] = 1e5
    perm, wt = P.encode(0, 0, w.ns)
    ctx.forward(v, perm, wt, [w.ns])
    assert ctx.device_status() == -2
    # The error word also stops the multi-step launch: its warps see it at
    # their next dependency wait, give up and drain their copies.  The
    # context stays usable, and the next call is bit-identical to a fresh
    # context's.
    v[0, 5, 5] = 2000.0
    d1 = ctx.forward(v, perm, wt, [w.ns])
    assert ctx.device_status() == 0
    d2 = make_ctx(P, w, 1).forward(v, perm, wt, [w.ns])
    assert torch.equal(d1, d2)


def test_all_step_kernel_variants_bit_identical(P, torch):
    # every compiled tile/ring variant performs the same per-point arithmetic
    w = synth.tiny2d(nz=50, nx=300, nt=120, ns=6, nr=30, nb=10)
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 40 + s, 1500, 2500)
                               for s in range(2)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 4)).cuda()
    perm, wt = P.encode(8, 1, w.ns)
    ctx = make_ctx(P, w, 6)
    ref = None
    nvar = len(ctx.variants()["forward_ms"])
    for fv in range(nvar):
        ctx.set_variants(fv, fv % 4)
        m, g = ctx.gradient(v, perm, wt, [3, 2, 1], d_obs, 1.0)
        info = ctx.variants()
        assert info["forward"] == fv and info["adjoint"] == fv % 4
        if ref is None:
            ref = (m.clone(), g.clone())
        else:
            assert torch.equal(m, ref[0]) and torch.equal(g, ref[1]), info
    ctx.set_variants(-1, -1)
    m, g = ctx.gradient(v, perm, wt, [3, 2, 1], d_obs, 1.0)
    info = ctx.variants()
    assert min(x for x in info["forward_ms"] if x > 0) > 0
    assert torch.equal(g, ref[1])


def test_chunked_gradient_bit_identical(P, torch):
    # a workspace too small for all samples at once makes fwi_gradient process
    # them in chunks; every sample's arithmetic is unchanged
    w = synth.tiny2d(nz=40, nx=70, nt=150, ns=4, nr=12, nb=6)
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 50 + s, 1500, 2500)
                               for s in range(3)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 6)).cuda()
    encs = [P.encode(4, s, w.ns) for s in range(3)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    big = make_ctx(P, w, 6, budget=1 << 30)
    m1, g1 = big.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    assert big.plan_info()["samples_per_chunk"] == 3
    field = (w.nz + 2 * w.nb + 8) * (((w.nx + 2 * w.nb + 8) + 31) // 32 * 32) * 4
    small = make_ctx(P, w, 6, budget=60 * 2 * field)
    m2, g2 = small.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    torch.cuda.synchronize()
    assert small.plan_info()["samples_per_chunk"] == 1
    assert torch.equal(g1, g2) and torch.equal(m1, m2)


def test_binding_rejects_mis_sized_buffers(P, torch):
    # sizes are checked on the host before the library is called
    w = synth.tiny2d(nt=50)
    ctx = make_ctx(P, w, 2)
    v = torch.full((1,) + w.shape, 2000.0, device="cuda")
    perm, wt = P.encode(1, 0, w.ns)
    d_obs = torch.zeros(w.ns, w.nt, w.nr, device="cuda")
    with pytest.raises(ValueError, match="d_obs"):
        ctx.gradient(v, perm, wt, [w.ns], d_obs[:, :-1], 1.0)
    with pytest.raises(ValueError, match="vel"):
        ctx.forward(v[:, :-1], perm, wt, [w.ns])
    with pytest.raises(ValueError, match="out"):
        ctx.forward(v, perm, wt, [w.ns], out=torch.empty(1, 1, w.nt, w.nr - 1, device="cuda"))
    with pytest.raises(ValueError, match="grad"):
        ctx.gradient(v, perm, wt, [w.ns], d_obs, 1.0, grad=torch.empty(2, *w.shape, device="cuda"))
    with pytest.raises(ValueError, match="d_cot"):
        ctx.adjoint(v, perm, wt, [w.ns], torch.zeros(1, 2, w.nt, w.nr, device="cuda"))
    with pytest.raises(ValueError, match="grad"):
        P.langevin_step(v, v[:, :-1].contiguous(), 1.0, 1.0, 0.0, 1e4, 1, 1)
    with pytest.raises(ValueError, match="x0"):
        P.renoise(v, v[:, :-1].contiguous(), 0.5, 0.6, 1 - 0.5 / 0.6, 1, 1)
    with pytest.raises(ValueError, match="out"):
        P.renoise(v, v, 0.5, 0.6, 1 - 0.5 / 0.6, 1, 1, out=torch.empty(3, device="cuda"))
    with pytest.raises(ValueError, match="grad"):
        ctx.langevin_precond(v, v[:, :-1].contiguous(), torch.zeros_like(v), 1, 1.0, 1.0, 0.0, 1e4, 1, 1)
    assert ctx.device_status() == 0


def test_degenerate_calls_are_rejected_and_leave_the_context_usable(P, torch):
    # empty batches, empty or oversized supergathers, shot ids outside the
    # geometry and weights other than +-1 are refused on the host
    # (FWI_ERR_ARG); the next valid call matches a fresh context bit for bit
    w = synth.tiny2d(nt=60)
    ctx = make_ctx(P, w, 2)
    v = torch.tensor(synth.models.random_smooth_model(w.shape, 3, 1500, 2500)[None]).cuda()
    perm, wt = P.encode(2, 0, w.ns)
    bad_calls = [
        lambda: ctx.forward(v[:0], perm, wt, [w.ns]),            # no samples
        lambda: ctx.forward(v, perm, wt, []),                    # no supergathers
        lambda: ctx.forward(v, perm, wt, [w.ns, 0]),             # an empty supergather
        lambda: ctx.forward(v, perm, wt, [w.ns, 1]),             # more shots than the geometry has
        lambda: ctx.forward(v, perm, wt, [1, 1, 1]),             # more wavefields than the context holds
        lambda: ctx.forward(v, np.array([0, 1, 2, w.ns], np.int32), wt, [w.ns]),   # shot id out of range
        lambda: ctx.forward(v, np.array([0, 1, 2, -1], np.int32), wt, [w.ns]),     # negative shot id
        lambda: ctx.forward(v, perm, np.array([1, -1, 0, 1], np.int8), [w.ns]),    # weight not +-1
    ]
    for i, call in enumerate(bad_calls):
        with pytest.raises(P.FwiError) as e:
            call()
        assert e.value.code == -1, (i, e.value.code)
    d = ctx.forward(v, perm, wt, [2, 2])
    fresh = make_ctx(P, w, 2)
    d_fresh = fresh.forward(v, perm, wt, [2, 2])
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    assert torch.equal(d, d_fresh)
