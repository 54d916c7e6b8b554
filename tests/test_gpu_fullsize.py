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
