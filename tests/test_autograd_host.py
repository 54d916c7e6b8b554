"""Host-side wiring of the autograd Functions (paper_2512_12797_gb300/autograd.py)
without a GPU: a fake context whose records are a fixed linear map of the
velocity stands in for the library, so the backward passes can be checked
against the exact transposed map.  The library's own forward, adjoint and
gradient calls are checked against the oracle in tests/test_gpu_autograd.py."""
import pytest
import torch

from paper_2512_12797_gb300 import autograd as AG


class FakeFWI:
    """records[s] = A vel[s] (reshaped [nsg][nt][nr]); misfit and gradient of
    scale * ||records - d||^2 / (2 sigma^2) with d the given target."""

    def __init__(self, phys, nsg=2, nt=3, nr=4, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.A = torch.randn(nsg * nt * nr, phys, generator=g, dtype=torch.float64)
        self.rshape = (nsg, nt, nr)

    def forward(self, vel, perm, w, sg):
        n = vel.shape[0]
        return (vel.reshape(n, -1).double() @ self.A.T).float().reshape((n,) + self.rshape)

    def adjoint(self, vel, perm, w, sg, d_cot):
        n = vel.shape[0]
        return (d_cot.reshape(n, -1).double() @ self.A).float().reshape(vel.shape)

    def gradient(self, vel, perm, w, sg, d_obs, sigma, scale):
        n = vel.shape[0]
        r = vel.reshape(n, -1).double() @ self.A.T - d_obs.reshape(1, -1).double()
        mis = scale * 0.5 * (r * r).sum(1) / sigma ** 2
        return mis, (scale * (r @ self.A) / sigma ** 2).float().reshape(vel.shape)


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(AG, "_check_vel", lambda v: None)  # the real check demands a CUDA tensor
    torch.manual_seed(1234)  # the tests' random inputs are the same on every run
    return FakeFWI(phys=5 * 6)


def test_records_backward_is_the_transposed_map(fake):
    vel = torch.randn(3, 5, 6, requires_grad=True)
    d = AG.encoded_records(fake, vel, None, None, [1, 1])
    cot = torch.randn(d.shape)
    (d * cot).sum().backward()
    expect = (cot.reshape(3, -1).double() @ fake.A).reshape(vel.shape)
    assert vel.grad.dtype == torch.float32
    assert torch.allclose(vel.grad.double(), expect, rtol=1e-5, atol=1e-5)


def test_misfit_backward_scales_each_sample_by_its_cotangent(fake):
    vel = torch.randn(2, 5, 6, requires_grad=True)
    d_obs = torch.randn(fake.rshape)
    phi = AG.encoded_misfit(fake, vel, None, None, [1, 1], d_obs, 0.5, 2.0)
    assert phi.dtype == torch.float64 and phi.shape == (2,)
    w = torch.tensor([3.0, -0.5], dtype=torch.float64)
    (gv,) = torch.autograd.grad((phi * w).sum(), vel)
    _, g = fake.gradient(vel.detach(), None, None, None, d_obs, 0.5, 2.0)
    assert torch.allclose(gv, g * w.float().view(-1, 1, 1), rtol=1e-6, atol=1e-6)


def test_misfit_gradient_matches_central_differences_of_the_fake(fake):
    vel = torch.randn(1, 5, 6, dtype=torch.float32, requires_grad=True)
    d_obs = torch.randn(fake.rshape)
    AG.encoded_misfit(fake, vel, None, None, [1, 1], d_obs, 1.0, 1.0).sum().backward()
    dv = torch.randn(vel.shape, dtype=torch.float64)
    eps = 1e-2
    v0 = vel.detach().double()
    fp = fake.gradient(v0 + eps * dv, None, None, None, d_obs, 1.0, 1.0)[0].item()
    fm = fake.gradient(v0 - eps * dv, None, None, None, d_obs, 1.0, 1.0)[0].item()
    dirn = float((vel.grad.double() * dv).sum())
    # the misfit is quadratic in vel, so the central difference (in FP64) is
    # exact up to rounding; vel.grad is FP32, the Function's output type, so
    # the bound is relative to |grad| |dv|, not to the directional derivative
    # (which a random dv can make small)
    assert abs((fp - fm) / (2 * eps) - dirn) < 1e-5 * float(vel.grad.double().norm() * dv.norm())


def test_misfit_refuses_differentiable_data(fake):
    vel = torch.randn(1, 5, 6, requires_grad=True)
    d_obs = torch.randn(fake.rshape, requires_grad=True)
    with pytest.raises(ValueError, match="d_obs"):
        AG.encoded_misfit(fake, vel, None, None, [1, 1], d_obs, 1.0)


def test_real_check_rejects_host_tensors():
    with pytest.raises(TypeError, match="CUDA"):
        AG._check_vel(torch.zeros(1, 2, 2))
