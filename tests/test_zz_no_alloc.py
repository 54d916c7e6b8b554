"""fwi_residual_misfit_noalloc: the encoded residual and misfit for callers
that cannot allocate device memory (plug-ins whose host application owns the
device memory pool, loops that cannot take the synchronisation an allocation
implies).  Its scratch is one static device array shared by all calls and
keeping the last call's contents, so these tests call it several times in a
row with different batch sizes (6, then 2, then 6 wavefields): a smaller call
after a larger one would expose stale partial sums or shot lists.  Each
result is checked against the allocating entry point fwi_gradient, and the
residual element by element against the oracle's encoded residual.  Collected
last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MISFIT_TOL = 1e-5   # relative, as in the other misfit parity checks
RHAT_TOL = 1e-6     # relative L2 of the FP32 residual against FP64


@pytest.fixture(scope="module")
def P():
    from paper_2512_12797_gb300 import build
    build.build()
    import paper_2512_12797_gb300 as P
    return P


CALLS = [(3, [3, 2], 0), (1, [2], 1), (2, [2, 2, 2], 2)]  # (nsamp, sg_sizes, encoding); B = 6, 2, 6


def _encoding(P, nsamp, ns, it):
    encs = [P.encode(5, it * 10 + s, ns) for s in range(nsamp)]
    return np.stack([e[0] for e in encs]), np.stack([e[1] for e in encs])


def test_noalloc_misfit_matches_fwi_gradient_on_consecutive_calls(P):
    import torch
    w = synth.tiny2d(nz=40, nx=140, nt=180, ns=6, nr=16, nb=8)
    ctx = P.FWI(w.grid_dict(), w.src, w.rec, 6, 1 << 28)
    d_obs = torch.tensor(synth.random_records(w, 3)).cuda()
    vs = torch.tensor(np.stack([synth.models.random_smooth_model(w.shape, 20 + s, 1500, 2500)
                                for s in range(3)])).cuda()
    for call, (nsamp, sg, it) in enumerate(CALLS):
        perm, wt = _encoding(P, nsamp, w.ns, it)
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


def test_noalloc_residual_matches_oracle_elementwise(P):
    """rhat and misfit against the oracle's FP64 encoded residual on seeded
    synthetic records, for consecutive calls of different sizes, one of them
    in place (rhat = d_pred) and one on a non-default stream."""
    import torch
    import oracle as O
    w = synth.tiny2d(nz=40, nx=140, nt=180, ns=6, nr=16, nb=8)
    d_obs_h = synth.random_records(w, 4)
    d_obs = torch.tensor(d_obs_h).cuda()
    sigma = 0.3
    side = torch.cuda.Stream()
    for call, (nsamp, sg, it) in enumerate(CALLS):
        perm, wt = _encoding(P, nsamp, w.ns, it)
        nsg = len(sg)
        d_pred_h = synth.random_records(w, 40 + call, nshots=nsamp * nsg).reshape(nsamp, nsg, w.nt, w.nr)
        ref_r = np.stack([(d_pred_h[s].astype(np.float64) - O.encoded_data(d_obs_h, perm[s], wt[s], sg))
                          / sigma ** 2 for s in range(nsamp)])
        scale = w.ns / sum(sg)
        ref_m = scale * 0.5 * sigma ** 2 * (ref_r ** 2).sum(axis=(1, 2, 3))
        d_pred = torch.tensor(d_pred_h).cuda()
        if call == 1:  # in place, on a side stream
            side.wait_stream(torch.cuda.current_stream())
            got, rhat = P.residual_misfit_noalloc(d_pred, d_obs, perm, wt, sg, sigma, rhat=d_pred, stream=side)
            side.synchronize()
            assert rhat.data_ptr() == d_pred.data_ptr()
        else:
            got, rhat = P.residual_misfit_noalloc(d_pred, d_obs, perm, wt, sg, sigma)
        torch.cuda.synchronize()
        r = rhat.double().cpu().numpy()
        rel = np.linalg.norm(r - ref_r) / np.linalg.norm(ref_r)
        assert rel < RHAT_TOL, (call, rel)
        m = got.cpu().numpy()
        assert np.all(np.abs(m - ref_m) / ref_m < MISFIT_TOL), (call, m, ref_m)


def test_noalloc_rejects_scratch_beyond_its_maximum(P):
    """A batch whose scratch exceeds FWI_NOALLOC_MAX_BYTES (1 MiB) is refused
    with FWI_ERR_ARG before any launch; one just under it runs."""
    import torch
    w = synth.tiny2d(nz=20, nx=40, nt=16, ns=6, nr=4, nb=4)
    d_obs = torch.tensor(synth.random_records(w, 5)).cuda()
    perm, wt = _encoding(P, 1, w.ns, 3)
    # scratch: 512 B of partial sums per wavefield plus the encoding and shot
    # lists, each piece rounded to 256 B: 1,010,688 B at 1700 wavefields,
    # 1,070,080 B at 1800
    ok = torch.zeros((1700, 1, w.nt, w.nr), device="cuda")
    misfit, _ = P.residual_misfit_noalloc(ok, d_obs, perm, wt, [6], 1.0)
    torch.cuda.synchronize()
    assert torch.isfinite(misfit).all()
    big = torch.zeros((1800, 1, w.nt, w.nr), device="cuda")
    with pytest.raises(P.FwiError) as e:
        P.residual_misfit_noalloc(big, d_obs, perm, wt, [6], 1.0)
    assert e.value.code == -1  # FWI_ERR_ARG
