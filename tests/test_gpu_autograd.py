"""Velocity as a differentiable PyTorch input: the autograd Functions over
fwi_forward / fwi_adjoint / fwi_gradient against the FP64 oracle's
transposed Jacobian and gradient, against central differences of the
device misfit, and checkpointed against stored wavefields.

Tolerances as the other parity tests: relative L2 <= 1e-5 on records and
<= 1e-4 on gradients.
"""
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


def _case(nsamp=2, lo=1500.0, hi=2500.0):
    w = synth.tiny2d(nz=40, nx=70, nt=300, ns=4, nr=12, nb=6)
    vel = np.stack([synth.models.random_smooth_model(w.shape, 20 + s, lo, hi) for s in range(nsamp)])
    encs = [O.encode(3 + s, 1, w.ns) for s in range(nsamp)]
    return w, vel, np.stack([e[0] for e in encs]), np.stack([e[1] for e in encs])


def test_records_backward_is_oracle_transposed_jacobian(P):
    import torch
    from paper_2512_12797_gb300.autograd import encoded_records
    w, vel, perm, wt = _case()
    sg = [3, 1]
    g = O.Grid.from_workload(w)
    fwi = P.FWI(w.grid_dict(), w.src, w.rec, len(vel) * len(sg), 1 << 30)
    v = torch.tensor(vel, device="cuda", requires_grad=True)
    d = encoded_records(fwi, v, perm, wt, sg)
    cot = synth.random_records(w, 5, nshots=len(vel) * len(sg)).reshape(d.shape)
    (d * torch.tensor(cot, device="cuda")).sum().backward()
    torch.cuda.synchronize()
    assert fwi.device_status() == 0
    assert v.grad.shape == v.shape and v.grad.dtype == torch.float32
    for s in range(len(vel)):
        ref_d = O.encoded_forward(g, vel[s], w.src, w.rec, perm[s], wt[s], sg)
        assert rel(d[s].detach().cpu().numpy(), ref_d) < FWD_TOL
        ref_g = O.records_vjp(g, vel[s], w.src, w.rec, perm[s], wt[s], sg, cot[s].astype(np.float64))
        e = rel(v.grad[s].cpu().numpy(), ref_g)
        assert e < GRAD_TOL, (s, e)


def test_misfit_backward_matches_oracle_and_central_differences(P):
    import torch
    from paper_2512_12797_gb300.autograd import encoded_misfit
    # models kept 20 m/s inside [vmin, vmax] = [1500, 2500]: the perturbed
    # copies below must not exceed the grid's velocity bound, which the
    # library refuses (FWI_ERR_CFL)
    w, vel, perm, wt = _case(lo=1520.0, hi=2480.0)
    sg, sigma = [2, 2], 0.5
    g = O.Grid.from_workload(w)
    truth = synth.models.random_smooth_model(w.shape, 4, 1500, 2500)
    d_obs = np.stack([O.forward_shot(g, truth, w.src[i:i + 1], [1.0], w.rec) for i in range(w.ns)])
    d_obs_d = torch.tensor(d_obs, dtype=torch.float32, device="cuda")
    fwi = P.FWI(w.grid_dict(), w.src, w.rec, len(vel) * len(sg), 1 << 30)
    v = torch.tensor(vel, device="cuda", requires_grad=True)
    phi = encoded_misfit(fwi, v, perm, wt, sg, d_obs_d, sigma)
    assert phi.dtype == torch.float64 and phi.shape == (len(vel),)
    weights = torch.tensor([1.0, 0.25], dtype=torch.float64, device="cuda")
    (phi * weights).sum().backward()
    grad = v.grad.double().cpu().numpy()
    for s in range(len(vel)):
        phi_ref, g_ref = O.gradient(g, vel[s], w.src, w.rec, d_obs, perm[s], wt[s], sg, sigma)
        assert abs(phi[s].item() - phi_ref) < 1e-5 * abs(phi_ref)
        e = rel(grad[s], weights[s].item() * g_ref)
        assert e < GRAD_TOL, (s, e)
    # central differences of the device misfit along a smooth direction
    dv = synth.models.random_smooth_model(w.shape, 9, -1.0, 1.0).astype(np.float64)
    eps = 5.0
    with torch.no_grad():
        vp = torch.tensor(vel + eps * dv, dtype=torch.float32, device="cuda")
        vm = torch.tensor(vel - eps * dv, dtype=torch.float32, device="cuda")
        step = (vp - vm).double().cpu().numpy()             # the FP32-rounded 2 eps dv
        fp = encoded_misfit(fwi, vp, perm, wt, sg, d_obs_d, sigma).cpu().numpy()
        fm = encoded_misfit(fwi, vm, perm, wt, sg, d_obs_d, sigma).cpu().numpy()
    assert fwi.device_status() == 0
    for s in range(len(vel)):
        dirn = float(np.sum(grad[s] / weights[s].item() * step[s]))
        assert abs((fp[s] - fm[s]) - dirn) < 2e-3 * abs(dirn), (s, fp[s] - fm[s], dirn)


def test_records_backward_checkpointed_is_bit_exact(P):
    # the adjoint re-runs the forward with checkpoints and recomputation when
    # the workspace cannot hold every wavefield; the result is bit-identical
    import torch
    from paper_2512_12797_gb300.autograd import encoded_records
    w, vel, perm, wt = _case(1)
    sg = [2, 2]
    field = (w.nz + 2 * w.nb + 8) * (((w.nx + 2 * w.nb + 8) + 31) // 32 * 32) * 4
    grads = []
    for budget in (1 << 30, 80 * 2 * field):
        fwi = P.FWI(w.grid_dict(), w.src, w.rec, 2, budget)
        v = torch.tensor(vel, device="cuda", requires_grad=True)
        d = encoded_records(fwi, v, perm, wt, sg)
        cot = torch.tensor(synth.random_records(w, 6, nshots=2).reshape(d.shape), device="cuda")
        (d * cot).sum().backward()
        torch.cuda.synchronize()
        grads.append((v.grad.clone(), fwi.plan_info()["recomputed_steps"]))
        fwi.close()
    assert grads[0][1] == 0 and grads[1][1] > 0
    assert torch.equal(grads[0][0], grads[1][0])


def test_misfit_drives_a_torch_optimizer(P):
    # vel as an nn.Parameter under torch.optim.Adam: the encoded misfit of a
    # fixed encoding decreases over a few steps
    import torch
    from paper_2512_12797_gb300.autograd import encoded_misfit
    w, vel, perm, wt = _case(1)
    g = O.Grid.from_workload(w)
    truth = synth.models.random_smooth_model(w.shape, 4, 1500, 2500)
    d_obs = torch.tensor(np.stack([O.forward_shot(g, truth, w.src[i:i + 1], [1.0], w.rec)
                                   for i in range(w.ns)]), dtype=torch.float32, device="cuda")
    fwi = P.FWI(w.grid_dict(), w.src, w.rec, 1, 1 << 30)
    v = torch.nn.Parameter(torch.tensor(vel, device="cuda"))
    opt = torch.optim.Adam([v], lr=5.0)
    hist = []
    for _ in range(6):
        opt.zero_grad()
        phi = encoded_misfit(fwi, v, perm, wt, [w.ns], d_obs, 1.0)
        phi.sum().backward()
        opt.step()
        hist.append(phi.item())
    assert fwi.device_status() == 0
    assert all(b < a for a, b in zip(hist, hist[1:])) and hist[-1] < 0.9 * hist[0], hist
