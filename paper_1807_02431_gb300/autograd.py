"""Reverse-mode differentiation through libgrp (not part of the paper; it serves fitting the force
field that drives the dynamics).

``potential_energy(sysh, q, theta)`` returns V(q_b; theta) of Eq. 1 for a batch of configurations; its
backward pass calls ``grp_energy_grad`` with the incoming cotangent as weights, so that the force
kernel gives dV/dq and the parameter kernel gives dV/d theta (theta = sigma_i, epsilon_i, dihedral k_t).

``segment_loss(rep, theta, k, ...)`` advances a replica set k Langevin steps and returns the time- and
replica-averaged loss g(O(q_t)) of the segment; its gradient with respect to theta comes from the
adjoint sweep of ``grp_adjoint_segment`` (noise held fixed), computed with the forward pass.

Every value is computed by the CUDA library; torch only holds the device buffers.
"""
from __future__ import annotations

import torch

from . import binding as B


def current_params(sysh: B.SystemHandle, device=None) -> torch.Tensor:
    """The system's parameters theta as a device FP64 tensor [n_theta]."""
    n = B.grp_param_count(sysh)
    th = torch.empty(n, dtype=torch.float64, device=device or torch.device("cuda"))
    if n:
        B.grp_get_params(sysh, th, torch.cuda.current_stream())
    return th


class _PotentialEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, theta, sysh):
        st = torch.cuda.current_stream()
        B.grp_set_params(sysh, theta, st)
        e = torch.empty(q.shape[0], dtype=torch.float64, device=q.device)
        B.grp_energy_grad(sysh, q.shape[0], q, None, e, None, None, st)
        ctx.save_for_backward(q, theta)
        ctx.sysh = sysh
        return e

    @staticmethod
    def backward(ctx, g):
        q, theta = ctx.saved_tensors
        st = torch.cuda.current_stream()
        B.grp_set_params(ctx.sysh, theta, st)
        gq = torch.empty_like(q) if ctx.needs_input_grad[0] else None
        gth = torch.empty_like(theta) if ctx.needs_input_grad[1] else None
        B.grp_energy_grad(ctx.sysh, q.shape[0], q, g.contiguous(), None, gq, gth, st)
        return gq, gth, None


def potential_energy(sysh: B.SystemHandle, q: torch.Tensor, theta: torch.Tensor | None = None) -> torch.Tensor:
    """V(q_b; theta) for q of shape [B, n, 3] or [n, 3] (FP64, CUDA); differentiable in q and theta.

    theta = None uses the system's current parameters (not differentiated).  Evaluating with a theta
    also makes it the system's parameters for later calls (dynamics included)."""
    if q.dtype != torch.float64 or not q.is_cuda:
        raise TypeError("q must be a CUDA float64 tensor")
    single = q.dim() == 2
    qb = (q.unsqueeze(0) if single else q).contiguous()
    if theta is None:
        theta = current_params(sysh, q.device)
    if theta.dtype != torch.float64 or not theta.is_cuda or theta.dim() != 1:
        raise TypeError("theta must be a 1-D CUDA float64 tensor")
    e = _PotentialEnergy.apply(qb, theta.contiguous(), sysh)
    return e[0] if single else e


class _SegmentLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, rep, k, t_gr, checkpoint, obs, transform, center, width):
        st = torch.cuda.current_stream()
        B.grp_set_params(rep.sysh, theta, st)
        g = torch.empty_like(theta)
        loss = B.grp_adjoint_segment(rep, k, t_gr, checkpoint, obs, transform, center, width, d_grad_theta=g,
                                     stream=st)
        ctx.save_for_backward(g)
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return (gout * g,) + (None,) * 8


def segment_loss(rep: B.ReplicasHandle, theta: torch.Tensor, k: int, t_gr: int, obs: int, transform: int = 0,
                 center: float = 0.0, width: float = 1.0, checkpoint: int = 100) -> torch.Tensor:
    """Loss of the next k steps of the replica set with force-field parameters theta (which become the
    system's), differentiable in theta; the replica set advances k steps."""
    if theta.dtype != torch.float64 or not theta.is_cuda or theta.dim() != 1:
        raise TypeError("theta must be a 1-D CUDA float64 tensor")
    return _SegmentLoss.apply(theta.contiguous(), rep, k, t_gr, checkpoint, obs, transform, center, width)
