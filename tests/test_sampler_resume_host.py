"""Checkpoint and resume of the encoded diffusion sampler, on the CPU: the
library's solve, Langevin and re-noise calls are replaced by small CPU fakes
with the same counter-based randomness, so the sampler's own bookkeeping
(levels, step counters, preconditioner state, histories) is what is tested.
A run stopped before a level, saved with torch.save and resumed must equal
the uninterrupted run bit for bit."""
import io

import numpy as np
import pytest
import torch

from paper_2512_12797_gb300 import sampler as S


class FakeCtx:
    """Gradient of a quadratic misfit whose weight depends on the encoding,
    so a wrong encoding counter changes the result."""
    ns = 6

    def gradient(self, z, perm, w, sg, d_obs, sigma, scale=0.0, grad=None):
        wsum = torch.tensor(np.asarray(w, np.float64).sum(1) + 0.1 * np.asarray(perm, np.float64)[:, 0],
                            dtype=z.dtype).view(-1, 1, 1)
        grad.copy_((z - d_obs) * (1.0 + 0.05 * wsum) / sigma ** 2)
        return None, grad

    def langevin_precond(self, z, grad, v, k, eta, nu, vmin, vmax, seed, counter, m=None, alpha=0.9, beta1=0.9,
                         eps=1e-2, stream=None):
        # the moment bookkeeping of the library call, on the CPU
        v.mul_(alpha).addcmul_(grad, grad, value=1 - alpha)
        vh = v / (1 - alpha ** k)
        d = grad
        if m is not None:
            m.mul_(beta1).add_(grad, alpha=1 - beta1)
            d = m / (1 - beta1 ** k)
        r = vh.reshape(vh.shape[0], -1).mean(1).sqrt().view(-1, 1, 1)
        G = 1.0 / (vh.sqrt() + eps * r)
        z.sub_(eta * G * d).add_(nu * G.sqrt() * _noise(seed, counter, z)).clamp_(vmin, vmax)
        return z


def _noise(seed, counter, like):
    g = torch.Generator().manual_seed((seed * 1000003 + counter) % (2 ** 63))
    return torch.randn(like.shape, generator=g, dtype=like.dtype)


def fake_renoise(x_t, x0, abar_t, abar_prev, beta_t, seed, counter, out=None, stream=None):
    c0 = np.sqrt(abar_prev) * beta_t / (1 - abar_t)
    ct = np.sqrt(1 - beta_t) * (1 - abar_prev) / (1 - abar_t)
    var = (1 - abar_prev) / (1 - abar_t) * beta_t
    return c0 * x0 + ct * x_t + np.sqrt(var) * _noise(seed, counter, x_t)


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(S, "renoise", fake_renoise)


def _run(**kw):
    v_init = torch.full((12, 16), 2500.0)
    truth = v_init + 100 * torch.sin(torch.arange(16.0))[None]
    args = dict(ctx=FakeCtx(), v_init=v_init, d_obs=truth, truth=truth, nsamp=3, sg_sizes=[2, 3], t_start=40,
                stride=7, K=3, eta=5.0, nu=2.0, vmin=1500.0, vmax=4500.0, sigma=1.0, seed=11)
    args.update(kw)
    return S.encoded_diffusion_sampler(**args)


@pytest.mark.parametrize("refine", ["langevin", "adam"])
def test_resumed_run_is_bit_identical(fakes, refine):
    full = _run(refine=refine)
    part = _run(refine=refine, stop_at=19)
    assert part["samples"] is None and part["state"]["t"] == 19
    buf = io.BytesIO()
    torch.save(part["state"], buf)
    buf.seek(0)
    state = torch.load(buf)
    rest = _run(refine=refine, state=state)
    assert torch.equal(rest["samples"], full["samples"])
    assert rest["rmse"] == full["rmse"] and rest["solves"] == full["solves"]


def test_resume_refuses_a_state_from_other_arguments(fakes):
    part = _run(stop_at=25)
    with pytest.raises(ValueError, match="other arguments"):
        _run(state=part["state"], K=2)


def test_state_keeps_the_step_counter(fakes):
    # resuming with the step counter reset would redraw the same encodings
    # and noise as the first levels and give a different result
    full = _run()
    part = _run(stop_at=19)
    st = dict(part["state"])
    st["it"] = 0
    assert not torch.equal(_run(state=st)["samples"], full["samples"])
