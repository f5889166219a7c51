"""torch.autograd binding of the density -> ghost -> force chain.

``chain_outputs(x, m, u, off)`` runs the neighbour-list step of an
:class:`~paper_2606_23891_b300.pipeline.Offload` on device tensors and returns
the accelerations a (n, 3) and du/dt (n,); their backward calls the
library's adjoint kernels: the vector-Jacobian product of the chain (density
sums, ghost update, force sums; h, v and the switches' coefficients held
fixed) with whatever upstream adjoints of a and du/dt the loss passes, as
gradients with respect to x, m and u.  Outputs of inactive particles are
constants of the step (their adjoints are dropped).  The backward reads the
state the forward left in the store (densities, the ghost's fields): run it
before the next forward on the same Offload.  The pair lists are not kept
for it: the backward rebuilds them from the store's positions and supports
(one list build) before the adjoint kernels run.
"""
from __future__ import annotations

import torch


class ChainOutputs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, m, u, off):
        off.import_device({"x": x.detach().to(torch.float64).contiguous(),
                           "mass": m.detach().to(torch.float32).contiguous(),
                           "u": u.detach().to(torch.float32).contiguous()})
        off.list_step()
        out = off.export_device(("a", "u_dt"))
        ctx.off = off
        ctx.dtypes = (x.dtype, m.dtype, u.dtype)
        return out["a"], out["u_dt"]

    @staticmethod
    def backward(ctx, ga, gudt):
        off = ctx.off
        n = off.n
        if ga is None:
            ga = torch.zeros((n, 3), dtype=torch.float32, device=off.device)
        if gudt is None:
            gudt = torch.zeros(n, dtype=torch.float32, device=off.device)
        gx, gm, gu = off.adjoint(ga, gudt)
        tx, tm, tu = ctx.dtypes
        return gx.to(tx), gm.to(tm), gu.to(tu), None


def chain_outputs(x, m, u, off):
    """(a, du/dt) of the list step with a backward through the library."""
    return ChainOutputs.apply(x, m, u, off)


def loss(x, m, u, off):
    """L = sum |a|^2 + sum (du/dt)^2 over active particles."""
    a, udt = chain_outputs(x, m, u, off)
    return (a.double() ** 2).sum() + (udt.double() ** 2).sum()
