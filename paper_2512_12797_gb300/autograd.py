"""Velocity as a differentiable PyTorch input (Sec. 2.1, adjoint-state gradient).

Two `torch.autograd.Function`s over the library's calls; both only marshal
arguments, the solves run in the library's kernels:

- `encoded_records(fwi, vel, perm, w, sg_sizes)` returns the encoded records
  F~_j(v) [nsamp][nsg][nt][nr] (fwi_forward).  Its backward applies the
  transposed Jacobian to the incoming record cotangent (fwi_adjoint).  The
  forward wavefields are not kept between the two calls: the backward re-runs
  the forward solve, storing or checkpointing its wavefields in the context's
  workspace, then runs the adjoint solve and the imaging condition.  The cost
  of a forward/backward pair is therefore two forward solves and one adjoint
  solve per supergather.
- `encoded_misfit(fwi, vel, perm, w, sg_sizes, d_obs, sigma, scale)` returns
  the encoded misfit [nsamp] (float64, fwi_gradient).  One library call forms
  the misfit and its gradient together, one forward and one adjoint solve per
  supergather (the count of Sec. 2.4).  The backward multiplies the stored
  gradient by the incoming cotangent.

Observed data, encodings and the context are not differentiable inputs.
"""
import torch

__all__ = ["EncodedRecords", "EncodedMisfit", "encoded_records", "encoded_misfit"]


def _check_vel(vel):
    if not vel.is_cuda or vel.dtype != torch.float32:
        raise TypeError("vel must be a float32 CUDA tensor of shape [nsamp, *grid]")


class EncodedRecords(torch.autograd.Function):
    """d_pred = F~(vel); backward: vel.grad = J^T d_cot (fwi_adjoint)."""

    @staticmethod
    def forward(ctx, vel, fwi, perm, w, sg_sizes):
        _check_vel(vel)
        v = vel.detach().contiguous()
        ctx.fwi, ctx.enc = fwi, (perm, w, sg_sizes)
        ctx.save_for_backward(vel)
        return fwi.forward(v, perm, w, sg_sizes)

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, d_cot):
        (vel,) = ctx.saved_tensors
        if not ctx.needs_input_grad[0]:
            return None, None, None, None, None
        g = ctx.fwi.adjoint(vel.detach().contiguous(), *ctx.enc, d_cot.detach().float().contiguous())
        return g, None, None, None, None


class EncodedMisfit(torch.autograd.Function):
    """misfit = scale * sum_j Phi~_j(vel); backward: vel.grad = cot * dmisfit/dvel."""

    @staticmethod
    def forward(ctx, vel, fwi, perm, w, sg_sizes, d_obs, sigma, scale):
        _check_vel(vel)
        if isinstance(d_obs, torch.Tensor) and d_obs.requires_grad:
            raise ValueError("encoded_misfit differentiates with respect to vel only; detach d_obs")
        misfit, grad = fwi.gradient(vel.detach().contiguous(), perm, w, sg_sizes, d_obs, sigma, scale)
        ctx.save_for_backward(grad)
        return misfit

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, cot):
        (grad,) = ctx.saved_tensors
        shape = (-1,) + (1,) * (grad.dim() - 1)
        return cot.to(grad.dtype).reshape(shape) * grad, None, None, None, None, None, None, None


def encoded_records(fwi, vel, perm, w, sg_sizes):
    """Encoded records [nsamp][nsg][nt][nr], differentiable in vel."""
    return EncodedRecords.apply(vel, fwi, perm, w, sg_sizes)


def encoded_misfit(fwi, vel, perm, w, sg_sizes, d_obs, sigma, scale=0.0):
    """Encoded misfit [nsamp] (float64), differentiable in vel; scale <= 0
    selects N_s / sum(sg_sizes) as in fwi_gradient."""
    return EncodedMisfit.apply(vel, fwi, perm, w, sg_sizes, d_obs, sigma, scale)
