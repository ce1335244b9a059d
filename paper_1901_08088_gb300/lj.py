"""Differentiable truncated-and-shifted Lennard-Jones energy over a qbvh list.

Eq. 1 of the paper (Sec. 1), shifted to zero at r_cut, evaluated by the
library's fused CUDA pass: one sweep over the neighbor list gives the
per-system energies, the forces and the gradients with respect to the
per-type-pair eps and sigma.  The backward pass scales those by the incoming
gradient in a second small kernel.  The neighbor list is treated as a
constant (it does not depend differentiably on the positions).
"""
from __future__ import annotations

import numpy as np
import torch

from .qbvh import NeighborList, check, qbvh_lj_backward, qbvh_lj_forward, qbvh_pack_positions

__all__ = ["LJEnergy", "lj_energy", "pack_positions"]


def pack_positions(xyz: torch.Tensor, types: torch.Tensor | None = None) -> torch.Tensor:
    """[n, 3] float32 (+ [n] int32 types) -> [n, 4] float32 layout the build reads."""
    xyz = xyz.detach().contiguous()
    out = torch.empty((xyz.shape[0], 4), dtype=torch.float32, device=xyz.device)
    t = None if types is None else types.to(torch.int32).contiguous()
    check(qbvh_pack_positions(xyz, t, out), "qbvh_pack_positions")
    return out


class LJEnergy(torch.autograd.Function):
    """U[k] of every system k; gradients flow to xyz, eps and sig.

    forward(xyz [n,3] f32, eps [T,T] f32, sig [T,T] f32, nl, pos4 [n,4], r_cut [T,T])
    """

    @staticmethod
    def forward(ctx, xyz, eps, sig, nl: NeighborList, pos4, r_cut):
        dev = xyz.device
        n, T, S = nl.n, nl.n_types, nl.n_sys
        eps_c = eps.detach().to(torch.float32).contiguous()
        sig_c = sig.detach().to(torch.float32).contiguous()
        U = torch.empty(S, dtype=torch.float64, device=dev)
        F = torch.empty((n, 3), dtype=torch.float32, device=dev)
        dE = torch.empty((S, T, T), dtype=torch.float64, device=dev)
        dS = torch.empty((S, T, T), dtype=torch.float64, device=dev)
        rc = np.asarray(r_cut, np.float32)
        if rc.ndim == 0:
            rc = np.full((T, T), rc, np.float32)
        check(qbvh_lj_forward(nl.h, pos4, eps_c, sig_c, rc, None, U, F, dE, dS), "qbvh_lj_forward")
        ctx.nl = nl
        ctx.save_for_backward(F, dE, dS)
        ctx.mark_non_differentiable(F)
        return U

    @staticmethod
    def backward(ctx, gU):
        F, dE, dS = ctx.saved_tensors
        nl = ctx.nl
        g = gU.detach().to(torch.float64).contiguous()
        T = nl.n_types
        gpos = torch.empty_like(F) if ctx.needs_input_grad[0] else None
        geps = torch.empty((T, T), dtype=torch.float32, device=F.device) if ctx.needs_input_grad[1] else None
        gsig = torch.empty((T, T), dtype=torch.float32, device=F.device) if ctx.needs_input_grad[2] else None
        check(qbvh_lj_backward(nl.h, g, F, dE, dS, gpos, geps, gsig), "qbvh_lj_backward")
        return gpos, geps, gsig, None, None, None


def lj_energy(nl: NeighborList, xyz: torch.Tensor, eps: torch.Tensor, sig: torch.Tensor, r_cut,
              types: torch.Tensor | None = None, pos4: torch.Tensor | None = None) -> torch.Tensor:
    """Per-system LJ energies [n_sys] (FP64) over the list held by ``nl``.

    ``nl`` must hold a list queried for these positions with list radii
    >= r_cut.  ``eps``/``sig`` are [T, T] tensors (each entry its own
    parameter; tie them symmetric in the caller if desired).
    """
    if pos4 is None:
        pos4 = pack_positions(xyz, types)
    return LJEnergy.apply(xyz, eps, sig, nl, pos4, r_cut)
