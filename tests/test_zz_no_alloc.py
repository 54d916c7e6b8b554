"""fwi_residual_misfit_noalloc: the encoded residual and misfit for callers
that cannot allocate device memory (inside a stream capture, inside a host
application that owns the device memory pool, or in loops that cannot take
the synchronisation an allocation implies).  Its scratch is one static device
array shared by all calls, so this test calls it twice in a row, with
different encodings and batch sizes, and checks each result against the
misfit that the allocating entry point fwi_gradient reports for the same
inputs.  Collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MISFIT_TOL = 1e-5   # relative, as in the other misfit parity checks


@pytest.fixture(scope="module")
def P():
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    return P


def test_noalloc_misfit_matches_fwi_gradient_on_two_calls(P):
    import torch
    w = synth.tiny2d(nz=40, nx=140, nt=180, ns=6, nr=16, nb=8)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, 6, 1 << 28)
    d_obs = torch.tensor(synth.random_records(w, 3)).cuda()
    vs = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 20 + s, 1500, 2500)
                                for s in range(3)])).cuda()
    for call, (nsamp, sg, it) in enumerate([(3, [3, 2], 0), (2, [2, 2, 2], 1)]):
        encs = [P.encode(5, it * 10 + s, w.ns) for s in range(nsamp)]
        perm = np.stack([e[0] for e in encs])
        wt = np.stack([e[1] for e in encs])
        v = vs[:nsamp].contiguous()
        d_pred = ctx.forward(v, perm, wt, sg)
        ref, _ = ctx.gradient(v, perm, wt, sg, d_obs, 0.7)
        got, rhat = P.residual_misfit_noalloc(d_pred, d_obs, perm, wt, sg, 0.7)
        torch.cuda.synchronize()
        e = (got - ref).abs() / ref.abs()
        assert float(e.max()) < MISFIT_TOL, (call, e)
        # the residual it returns is the one the misfit sums
        scale = w.ns / sum(sg)
        phi = scale * 0.5 * (rhat.double() * 0.49).pow(2).sum(dim=(1, 2, 3)) / 0.49
        assert float(((phi - got).abs() / got.abs()).max()) < MISFIT_TOL
