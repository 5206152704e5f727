"""torch.autograd.Function wrappers over the library's hand-written adjoints.

Each forward and backward is one call into libmm_gb300.so (the checkpointed
reverse sweep of a trajectory included); this module only moves tensors.

* ``DemagField.apply(m, Ms_cell, ctx)``      H_demag(m), gradients to m and Ms
* ``ExchangeField.apply(m, Ms_cell, ctx)``   H_ex(m), gradients to m and Ms
* ``LLGStep.apply(m, Ms_cell, ctx, dt)``       one RK4 step of the LLG
  equation (Eq. 1), gradients to m and Ms
* ``RK4Trajectory.apply(m0, Ms_cell, ctx, dt, nsteps, checkpoint_every)``
  the state after ``nsteps`` RK4 steps of the LLG equation, gradients to m0
  and the per-cell Ms (sqrt(T) checkpointing inside the library).

``Ms_cell`` ([nz, ny, nx], the context's dtype) becomes the context's per-cell
Ms for the call.
"""

import torch

from . import (MM_RK4, mm_demag_field, mm_demag_vjp, mm_exchange_field, mm_exchange_vjp, mm_llg_step,
               mm_rk4_step_vjp, mm_rk4_trajectory, mm_rk4_trajectory_vjp, mm_set_material_fields)


class DemagField(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m, Ms_cell, mmctx):
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        m = m.detach().contiguous()
        H = torch.empty_like(m)
        mm_demag_field(mmctx, m, H)
        fctx.save_for_backward(m, Ms_cell)
        fctx.mmctx = mmctx
        return H

    @staticmethod
    def backward(fctx, gH):
        m, Ms_cell = fctx.saved_tensors
        mmctx = fctx.mmctx
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        gm = torch.empty_like(m)
        gMs = torch.zeros_like(Ms_cell)
        mm_demag_vjp(mmctx, gH.contiguous(), m, gm, gMs)
        return gm, gMs, None


class ExchangeField(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m, Ms_cell, mmctx):
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        m = m.detach().contiguous()
        H = torch.empty_like(m)
        mm_exchange_field(mmctx, m, H)
        fctx.save_for_backward(m, Ms_cell)
        fctx.mmctx = mmctx
        return H

    @staticmethod
    def backward(fctx, gH):
        m, Ms_cell = fctx.saved_tensors
        mmctx = fctx.mmctx
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        gm = torch.empty_like(m)
        gMs = torch.zeros_like(Ms_cell)
        mm_exchange_vjp(mmctx, gH.contiguous(), m, gm, gMs)
        return gm, gMs, None


class LLGStep(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m, Ms_cell, mmctx, dt):
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        m = m.detach().contiguous()
        out = m.clone()
        mm_llg_step(mmctx, out, 0.0, dt, MM_RK4)
        fctx.save_for_backward(m, Ms_cell)
        fctx.mmctx, fctx.dt = mmctx, dt
        return out

    @staticmethod
    def backward(fctx, gm):
        m, Ms_cell = fctx.saved_tensors
        mmctx = fctx.mmctx
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        lam = gm.detach().contiguous().clone()
        gMs = torch.zeros_like(Ms_cell)
        mm_rk4_step_vjp(mmctx, m, fctx.dt, lam, gMs)
        return lam, gMs, None, None


class RK4Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, m0, Ms_cell, mmctx, dt, nsteps, checkpoint_every=0):
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        m0 = m0.detach().contiguous()
        m = m0.clone()
        mm_rk4_trajectory(mmctx, m, dt, nsteps)
        fctx.save_for_backward(m0, Ms_cell)
        fctx.mmctx, fctx.dt, fctx.nsteps, fctx.chk = mmctx, dt, nsteps, checkpoint_every
        return m

    @staticmethod
    def backward(fctx, gm):
        m0, Ms_cell = fctx.saved_tensors
        mmctx = fctx.mmctx
        mm_set_material_fields(mmctx, Ms_cell.detach().contiguous())
        lam = gm.detach().contiguous().clone()
        gMs = torch.zeros_like(Ms_cell)
        mm_rk4_trajectory_vjp(mmctx, m0, fctx.dt, fctx.nsteps, lam, gMs, fctx.chk)
        return lam, gMs, None, None, None, None
