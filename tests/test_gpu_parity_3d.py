"""Parity of the 3D CUDA path (2.5D z-marching kernels) with the FP64 oracle.

Same tolerances as the 2D tests: relative L2 <= 1e-5 on records, <= 1e-4 on
the velocity gradient; checkpointed and stored gradients bit-identical.
Grids are chosen so that x and y tiles are ragged (padded extents not
multiples of 128 and 8).
"""
import numpy as np
import pytest

import oracle as O
import synth
from synth.workloads import Workload

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


def medium3d(nt=200, ns=4):
    nz, ny, nx, h = 48, 61, 70, 20.0
    src = np.array([[1, 12 + 10 * i, 10 + 15 * i] for i in range(ns)], np.int32)
    rec = np.array([[2, y, x] for y in range(3, ny, 7) for x in range(2, nx, 6)], np.int32)
    return Workload("medium3d", 3, nz, ny, nx, h, h, h, 10, 2e-3, nt, 8.0, 1500.0, 3500.0, src, rec,
                    [ns], 1, 11)


def test_forward_3d_tiny_matches_oracle(P):
    import torch
    w = synth.tiny3d(nt=120)
    g = O.Grid.from_workload(w)
    v = synth.models.random_smooth_model(w.shape, 2, 1500, 2500)
    perm, wt = P.encode(4, 2, w.ns)
    ref = O.encoded_forward(g, v, w.src, w.rec, perm, wt, [w.ns])
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, 1, 1 << 28)
    d = ctx.forward(torch.tensor(v[None]).cuda(), perm, wt, [w.ns])
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    e = rel(d[0].cpu().numpy(), ref)
    assert e < FWD_TOL, e


def test_forward_3d_medium_matches_oracle(P):
    import torch
    w = medium3d()
    g = O.Grid.from_workload(w)
    v = synth.models.layered_fault_3d(w.nz, w.ny, w.nx, 3, 1500.0, 3500.0)
    perm, wt = P.encode(6, 0, w.ns)
    ref = O.encoded_forward(g, v, w.src, w.rec, perm, wt, [2, 2])
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, 2, 1 << 30)
    d = ctx.forward(torch.tensor(v[None]).cuda(), perm, wt, [2, 2])
    e = rel(d[0].cpu().numpy(), ref)
    assert e < FWD_TOL, e


@pytest.mark.parametrize("sg,adj_variant", [([3, 1], -1), ([3, 1], 4), ([2, 1, 1], -1)])
def test_gradient_3d_batched_matches_oracle(P, sg, adj_variant):
    # adj_variant 4: the adjoint on pair tiles (two supergathers per CTA, one
    # imaging accumulator per pair); -1: autotuned, one-wavefield tiles
    import torch
    w = medium3d(nt=150)
    g = O.Grid.from_workload(w)
    nsamp = 2
    vs = np.stack([synth.models.random_smooth_model(w.shape, 30 + s, 1500, 3000) for s in range(nsamp)])
    d_obs = synth.random_records(w, 8)
    encs = [P.encode(2, s, w.ns) for s in range(nsamp)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, nsamp * len(sg), 1 << 31)
    ctx.set_variants(-1, adj_variant)
    mis, grad = ctx.gradient(torch.tensor(vs).cuda(), perm, wt, sg, torch.tensor(d_obs).cuda(), 0.3)
    assert ("pairs" in ctx.variants()["adjoint_name"]) == (adj_variant >= 4)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    for s in range(nsamp):
        phi, gref = O.gradient(g, vs[s], w.src, w.rec, d_obs, perm[s], wt[s], sg, 0.3)
        e_phi = abs(mis[s].item() - phi) / abs(phi)
        e_g = rel(grad[s].cpu().numpy(), gref)
        assert e_phi < 1e-5 and e_g < GRAD_TOL, (s, e_phi, e_g)


def test_gradient_3d_tiny_physical_data(P):
    import torch
    w = synth.tiny3d(nt=150)
    g = O.Grid.from_workload(w)
    truth = synth.models.random_smooth_model(w.shape, 4, 1500, 2500)
    v = synth.models.random_smooth_model(w.shape, 5, 1500, 2500)
    d_obs = np.stack([O.forward_shot(g, truth, w.src[i:i + 1], [1.0], w.rec) for i in range(w.ns)])
    perm, wt = P.encode(1, 3, w.ns)
    phi, gref = O.gradient(g, v, w.src, w.rec, d_obs, perm, wt, [w.ns], 1e-3)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, 1, 1 << 28)
    mis, grad = ctx.gradient(torch.tensor(v[None]).cuda(), perm, wt, [w.ns],
                             torch.tensor(d_obs, dtype=torch.float32).cuda(), 1e-3)
    e_phi = abs(mis.item() - phi) / abs(phi)
    e_g = rel(grad[0].cpu().numpy(), gref)
    assert e_phi < 1e-5 and e_g < GRAD_TOL, (e_phi, e_g)


def test_checkpointed_gradient_3d_bit_exact(P):
    import torch
    w = medium3d(nt=120)
    v = torch.tensor(synth.models.random_smooth_model(w.shape, 7, 1500, 3000)[None]).cuda()
    d_obs = torch.tensor(synth.random_records(w, 9)).cuda()
    perm, wt = P.encode(3, 3, w.ns)
    big = P.FWI(w.grid_dict(), w.src, w.rec, 2, 1 << 31)
    m1, g1 = big.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    nzp, nyp, nxp = w.nz + 20, w.ny + 20, w.nx + 20
    field = (nzp + 8) * (nyp + 8) * ((nxp + 8 + 31) // 32 * 32) * 4
    small = P.FWI(w.grid_dict(), w.src, w.rec, 2, 40 * 2 * field)
    m2, g2 = small.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    torch.cuda.synchronize()
    assert big.plan_info()["recomputed_steps"] == 0
    assert small.plan_info()["recomputed_steps"] > 0
    assert torch.equal(g1, g2) and torch.equal(m1, m2)


def test_chunked_gradient_3d_bit_identical(P):
    # a workspace too small for all samples' checkpoint plans at once makes
    # fwi_gradient process the 3D batch in chunks of one sample; every
    # sample's arithmetic is unchanged, so the results are bit-identical
    import torch
    w = medium3d(nt=120)
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 60 + s, 1500, 3000)
                               for s in range(3)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 10)).cuda()
    encs = [P.encode(6, s, w.ns) for s in range(3)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    big = P.FWI(w.grid_dict(), w.src, w.rec, 6, 1 << 32)
    m1, g1 = big.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    assert big.plan_info()["samples_per_chunk"] == 3
    nzp, nyp, nxp = w.nz + 20, w.ny + 20, w.nx + 20
    field = (nzp + 8) * (nyp + 8) * ((nxp + 8 + 31) // 32 * 32) * 4
    # 60 slots of one sample's two wavefields: 30 slots for two samples, fewer
    # than any plan for 120 steps needs
    small = P.FWI(w.grid_dict(), w.src, w.rec, 6, 60 * 2 * field)
    m2, g2 = small.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
    torch.cuda.synchronize()
    assert small.plan_info()["samples_per_chunk"] == 1
    assert small.plan_info()["recomputed_steps"] > 0
    assert torch.equal(g1, g2) and torch.equal(m1, m2)


def test_3d_step_variants_bit_identical(P):
    # the autotuner's 3D variants (CTA order; one or two z levels per march
    # step; for the forward, 64 x 16 tiles or 64 x 8 pair tiles) change only
    # which CTA runs which tile when and how a thread's instructions
    # interleave, not any point's arithmetic, so forced choices give
    # bit-identical records and gradients
    import torch
    w = medium3d(nt=60)
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 70 + s, 1500, 3000)
                               for s in range(2)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 11)).cuda()
    encs = [P.encode(8, s, w.ns) for s in range(2)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    out = []
    # adjoint on 64 x 16 tiles; bit 3: persistent grid; bit 4 (with bit 3): one multi-step launch per phase
    for var in ((0, 0), (1, 1), (2, 3), (3, 2), (4, 0), (7, 1), (5, 2), (6, 3), (11, 9), (12, 10), (15, 11),
                (25, 27), (30, 24),
                (8, 8)):
        ctx = P.FWI(w.grid_dict(), w.src, w.rec, 4, 1 << 31)
        ctx.set_variants(*var)
        m, g = ctx.gradient(v, perm, wt, [2, 2], d_obs, 1.0)
        rec = ctx.forward(v, perm, wt, [2, 2])
        out.append((m, g, rec))
        got = ctx.variants()
        assert (got["forward"], got["adjoint"]) == var
        assert ("pairs" in got["forward_name"]) == bool(var[0] & 4)
        assert ("persistent" in got["forward_name"]) == bool(var[0] & 8)
        assert ("multi-step" in got["forward_name"]) == bool(var[0] & 16)
        ctx.close()
    torch.cuda.synchronize()
    for m, g, rec in out[1:]:
        assert torch.equal(g, out[0][1]) and torch.equal(m, out[0][0]) and torch.equal(rec, out[0][2])


def wide3d(nt=60, ns=4):
    # a wide, shallow grid: 36 x 140 x 270 padded points, 5 x 9 = 45 tiles of
    # 64 x 16 per wavefield
    nz, ny, nx, h = 16, 120, 250, 20.0
    src = np.array([[1, 20 + 25 * i, 30 + 55 * i] for i in range(ns)], np.int32)
    rec = np.array([[2, y, x] for y in range(3, ny, 9) for x in range(2, nx, 11)], np.int32)
    return Workload("wide3d", 3, nz, ny, nx, h, h, h, 10, 2e-3, nt, 8.0, 1500.0, 3500.0, src, rec, [ns], 1, 11)


def test_3d_multistep_launch_many_columns_bit_identical(P):
    # 2 samples x 4 supergathers of one shot on the wide grid: 45 tiles x 4
    # wavefields = 180 columns per sample, more than one per SM in every
    # launch however the samples are chunked, so a CTA of a multi-step launch
    # runs several columns per step and waits on other CTAs' columns through
    # the progress flags; records and gradients must equal those of the
    # one-launch-per-step variants bit for bit (sources, receivers and
    # checkpoint segments)
    import torch
    w = wide3d()
    nsamp, sg = 2, [1, 1, 1, 1]
    tiles = -(-(w.nx + 2 * w.nb) // 64) * -(-(w.ny + 2 * w.nb) // 16)
    assert tiles * len(sg) > 152
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 90 + s, 1500, 3000)
                               for s in range(nsamp)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 13)).cuda()
    encs = [P.encode(10, s, w.ns) for s in range(nsamp)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    out = []
    for var in ((1, 0), (25, 24), (27, 25), (24, 9)):
        ctx = P.FWI(w.grid_dict(), w.src, w.rec, len(sg) * nsamp, 1 << 30)
        ctx.set_variants(*var)
        m, g = ctx.gradient(v, perm, wt, sg, d_obs, 1.0)
        rec = ctx.forward(v, perm, wt, sg)
        out.append((m, g, rec))
        got = ctx.variants()
        assert ("multi-step" in got["forward_name"]) == bool(var[0] & 16)
        assert ("multi-step" in got["adjoint_name"]) == bool(var[1] & 16)
        ctx.close()
    torch.cuda.synchronize()
    for m, g, rec in out[1:]:
        assert torch.equal(g, out[0][1]) and torch.equal(m, out[0][0]) and torch.equal(rec, out[0][2])


def test_3d_pair_tile_adjoint_variants_bit_identical(P):
    # the pair-tile adjoint's CTA orders and march forms agree bit for bit,
    # and with the 64 x 16 adjoint to FP32 rounding (another summation order
    # of the imaging term)
    import torch
    w = medium3d(nt=60)
    v = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 80 + s, 1500, 3000)
                               for s in range(2)])).cuda()
    d_obs = torch.tensor(synth.random_records(w, 12)).cuda()
    encs = [P.encode(9, s, w.ns) for s in range(2)]
    perm = np.stack([e[0] for e in encs])
    wt = np.stack([e[1] for e in encs])
    out = []
    for var in ((3, 4), (0, 5), (1, 6), (2, 7), (11, 12), (3, 13), (27, 28), (3, 0)):
        ctx = P.FWI(w.grid_dict(), w.src, w.rec, 4, 1 << 31)
        ctx.set_variants(*var)
        out.append(ctx.gradient(v, perm, wt, [2, 2], d_obs, 1.0))
        assert ("pairs" in ctx.variants()["adjoint_name"]) == bool(var[1] & 4)
        ctx.close()
    torch.cuda.synchronize()
    for m, g in out[1:7]:
        assert torch.equal(g, out[0][1]) and torch.equal(m, out[0][0])
    m0, g0 = out[7]
    assert torch.equal(m0, out[0][0])
    assert float((g0 - out[0][1]).norm() / g0.norm()) < 1e-6
