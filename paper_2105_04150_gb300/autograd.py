"""torch.autograd.Function around the hand-written adjoint (pd_adjoint_*).

``PeridynamicRun.apply(c_bond, load, u0, v0, model, n_steps, checkpoint_every)``
runs ``n_steps`` steps of ``model`` (an FP64 or PD_PREC_DW
``paper_2105_04150_gb300.Model``, with either integrator) from (u0, v0) with the
bond flags frozen, with the per-directed-bond stiffness ``c_bond`` and
body-force scale ``load``, and returns the final displacement u^N (n x 3).  Its backward runs the library's
reverse sweep and returns dL/dc_bond, dL/dload, dL/du0 and dL/dv0.

All arithmetic happens in the CUDA library; this module only moves tensors
in and out of the C ABI (CPU float64 tensors).
"""
from __future__ import annotations

import numpy as np
import torch

from . import pd_adjoint_backward, pd_adjoint_forward


class PeridynamicRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c_bond, load, u0, v0, model, n_steps, checkpoint_every=0):
        info = model.info()
        c_np = c_bond.detach().cpu().double().numpy()
        model.set_params(float(model.c_ref), float(model.sc_ref), float(load), model.rate_ref,
                         c_np)
        model.set_state(u0.detach().cpu().double().numpy(), v0.detach().cpu().double().numpy(),
                        step=model.step0_ref)
        model.set_bonds(model.bonds0_ref)
        pd_adjoint_forward(model.h, n_steps, checkpoint_every)
        u, _ = model.state()
        ctx.model = model
        ctx.n = info["n"]
        return torch.from_numpy(u)

    @staticmethod
    def backward(ctx, grad_u):
        g = grad_u.detach().cpu().double().contiguous().numpy()
        gc, gl, gu0, gv0 = pd_adjoint_backward(ctx.model.h, g)
        return (torch.from_numpy(gc), torch.tensor(gl, dtype=torch.float64),
                torch.from_numpy(gu0), torch.from_numpy(gv0), None, None, None)


def prepare(model, c_ref: float, sc_ref: float, rate_ref: float, step0: int = 0):
    """Record the constant parameters and reference bond flags the runs start from."""
    model.c_ref = c_ref
    model.sc_ref = sc_ref
    model.rate_ref = rate_ref
    model.step0_ref = step0
    model.bonds0_ref = np.array(model.bonds(), copy=True)
    return model
