"""Reverse-mode differentiation of simulations through the library's adjoint.

``rollout(sim, rho, u_r, u_theta, T, n_steps)`` sets f = f^eq of the given
fields (Eq. 10), advances ``n_steps`` steps of Eq. (38) and returns the fields
(rho, u_r, u_theta, T) of the final state (Eqs. 3-5).  It is differentiable
with respect to the initial fields: the backward pass runs the library's
adjoint step (pclb_adjoint_state) in reverse with sqrt(N) checkpointing --
checkpoints every ``segment`` steps on the forward pass, each segment's states
recomputed on the backward pass straight into the buffers the adjoint steps
read (pclb_step_states) -- and ends with the adjoint of the
equilibrium initialisation (pclb_set_state_vjp).  Checkpoints can live in
device memory or in page-locked host memory (``offload="host"``), which lets
the 2.2 GB states of a 4096 x 4096 run use the host's memory.

The workload objectives used with it (the paper defines none):
  * ``rm_mixing_width``: W = sum_r dr 4 c (1 - c), c(r) the azimuthal mean of
    (rho - rho_lo) / (rho_hi - rho_lo);
  * ``kh_vorticity_thickness``: delta = 2 U0 / max_r |d<u_theta>_theta / dr|;
and the initial conditions of the RM and KH workloads as torch functions of
their parameters (interface amplitudes a_k, shear amplitude U0).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import inputs as _inputs


def _store(buf: torch.Tensor, offload: str):
    if offload == "host":
        h = torch.empty(buf.shape, dtype=buf.dtype, pin_memory=True)
        h.copy_(buf, non_blocking=True)
        return h
    return buf


def _restore(buf: torch.Tensor, device) -> torch.Tensor:
    if buf.device.type == "cpu":
        return buf.to(device, non_blocking=True)
    return buf


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, u_r, u_t, T, sim, n_steps, segment, offload):
        n_steps = int(n_steps)
        seg = int(segment) if segment else max(1, int(math.ceil(math.sqrt(max(n_steps, 1)))))
        sim.set_state(rho.detach(), u_r.detach(), u_t.detach(), T.detach())
        ckpts = []
        done = 0
        while done < n_steps:
            ckpts.append(_store(sim.save_state(), offload))
            k = min(seg, n_steps - done)
            sim.step(k)
            done += k
        final = sim.save_state()
        outs = sim.moments()
        ctx.sim, ctx.n, ctx.seg, ctx.ckpts, ctx.final = sim, n_steps, seg, ckpts, final
        ctx.save_for_backward(rho, u_r, u_t, T)
        return outs

    @staticmethod
    def backward(ctx, g_rho, g_ur, g_ut, g_T):
        sim = ctx.sim
        rho, u_r, u_t, T = ctx.saved_tensors
        sim.load_state(ctx.final)
        sim.moments_vjp(*[None if g is None else g.contiguous() for g in (g_rho, g_ur, g_ut, g_T)])
        pool = []
        starts = list(range(0, ctx.n, ctx.seg))
        for si in reversed(range(len(starts))):
            k = min(ctx.seg, ctx.n - starts[si])
            first = _restore(ctx.ckpts[si], sim.device)  # f at the segment start
            while len(pool) < k - 1:
                pool.append(sim.new_state())
            states = [first] + pool[:k - 1]
            for j in range(1, k):                        # recompute the segment in place
                sim.step_states(states[j - 1], states[j])
            for j in reversed(range(k)):
                sim.adjoint_state(states[j])             # lam <- J(f_j)^T lam
            sim.sync()                                   # the segment's buffers are reused next
        grads = sim.set_state_vjp(rho.detach(), u_r.detach(), u_t.detach(), T.detach())
        ctx.ckpts = None
        return (*grads, None, None, None, None)


def rollout(sim, rho, u_r, u_theta, T, n_steps: int, segment: Optional[int] = None, offload: str = "device"):
    """Differentiable run of ``n_steps`` steps from f^eq(fields); returns the
    final (rho, u_r, u_theta, T) as device tensors of the context's dtype."""
    cast = [x.to(device=sim.device, dtype=sim.dtype).contiguous() for x in (rho, u_r, u_theta, T)]
    return _Rollout.apply(*cast, sim, n_steps, segment, offload)


# ---------------------------------------------------------------------------
# Objectives
# ---------------------------------------------------------------------------
def rm_mixing_width(rho: torch.Tensor, dr: float, rho_lo: float, rho_hi: float) -> torch.Tensor:
    """W = sum_r dr 4 c(r) (1 - c(r)), c = <(rho - rho_lo)/(rho_hi - rho_lo)>_theta."""
    c = ((rho - rho_lo) / (rho_hi - rho_lo)).mean(dim=0)
    return (4.0 * c * (1.0 - c)).sum() * dr


def kh_vorticity_thickness(u_theta: torch.Tensor, dr: float, u0: float) -> torch.Tensor:
    """delta_omega = 2 U0 / max_r |d<u_theta>/dr| (centred differences)."""
    m = u_theta.mean(dim=0)
    grad = (m[2:] - m[:-2]) / (2.0 * dr)
    return 2.0 * u0 / grad.abs().max()


# ---------------------------------------------------------------------------
# Initial conditions as torch functions of their parameters
# ---------------------------------------------------------------------------
def _mesh(w, device, dtype):
    r = torch.as_tensor(_inputs.radii(w.n_r, w.r_in, w.r_out), device=device, dtype=dtype)
    th = torch.as_tensor(_inputs.angles(w.n_theta, w.n_dirs, w.n_f), device=device, dtype=dtype)
    TH, R = torch.meshgrid(th, r, indexing="ij")
    return R, TH


def rm_fields(w, a: torch.Tensor, rho_in: float = 3.0, rho_out: float = 1.0, p0: float = 1.0,
              r_shock: float = 2.6, mach: float = 2.0, width_cells: float = 2.0, background: float = 0.0):
    """Fields of the RM workload with interface r = 2 + sum_k a_k cos(k theta)
    (the same construction as ``inputs.rm_adj``), differentiable in ``a``."""
    R, TH = _mesh(w, a.device, a.dtype)
    k = torch.arange(1, a.numel() + 1, device=a.device, dtype=a.dtype)
    r_if = 2.0 + (torch.cos(TH[..., None] * k) * a).sum(-1)
    dr = (w.r_out - w.r_in) / (w.n_r - 1)
    chi = 0.5 * (1.0 - torch.tanh((R - r_if) / (width_cells * dr)))
    rho = rho_out + (rho_in - rho_out) * chi
    T = p0 / rho
    rho_h, u_h, p_h, _ = _inputs.hugoniot_from_mach(rho_out, 0.0, p0, mach, direction=-1.0)
    post = R >= r_shock
    rho = torch.where(post, torch.full_like(rho, rho_h), rho)
    T = torch.where(post, torch.full_like(T, p_h / rho_h), T)
    u_r = torch.where(post, torch.full_like(rho, u_h), torch.zeros_like(rho))
    if background:
        m = 1.0 + background * torch.sin(3.0 * TH + 1.7 * R) * torch.cos(2.3 * R - TH)
        rho = rho * m
        T = T * m
    return rho, u_r, torch.zeros_like(rho), T


def kh_fields(w, u0: torch.Tensor):
    """Fields of the KH workload, differentiable in the shear amplitude u0."""
    R, TH = _mesh(w, u0.device, u0.dtype)
    s = torch.tanh((R - 2.0) / 0.02)
    rho = 1.5 + 0.5 * s
    u_t = u0 * s
    u_r = 0.01 * torch.sin(16.0 * TH) * torch.exp(-((R - 2.0) / 0.05) ** 2)
    return rho, u_r, u_t, 1.0 / rho
