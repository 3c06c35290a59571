"""torch.autograd.Function around the near-field forces and their adjoint.

forward:  pos (n, 4) float32 CUDA tensor of cell-relative offsets (cell
          widths, storage order of the box) -> accelerations (n, 4) float32
          in box units, computed by nf_set_particles + nf_forces.
backward: grad_acc -> grad_pos via nf_vjp (the hand-written adjoint kernel),
          times the cell width w because pos is in cell widths.

Cell membership is held fixed (the near field is discontinuous when a
particle changes cell), and the offsets are rounded to the library's 2^-22
grid in the forward pass; the gradient is that of the unrounded map.
backward refuses (RuntimeError) when the box's particles changed after the
forward pass (nf_generation), since the adjoint reads the box's current
positions.
"""
from __future__ import annotations

import torch

from . import NearField


class NearFieldForces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, box: NearField, cell_offsets, counts):
        box.set_stream(torch.cuda.current_stream())
        box.set_particles(cell_offsets, counts, pos.detach().contiguous())
        acc = torch.empty_like(pos)
        box.forces(acc)
        ctx.box = box
        ctx.generation = box.generation
        return acc

    @staticmethod
    def backward(ctx, grad_acc):
        box = ctx.box
        if box.generation != ctx.generation:
            raise RuntimeError("the box's particles changed between forward and backward (a load or "
                               "kick-drift ran in between); the adjoint would be that of other positions")
        box.set_stream(torch.cuda.current_stream())
        w = grad_acc.detach().contiguous().clone()
        w[:, 3] = 0
        g = torch.empty_like(w)
        box.vjp(w, g)
        g = g * (box.box / box.cpd)
        g[:, 3] = 0
        return g, None, None, None


def nearfield_forces(pos, box: NearField, cell_offsets, counts):
    """Differentiable near-field accelerations of `pos` (see module docstring)."""
    return NearFieldForces.apply(pos, box, cell_offsets, counts)
