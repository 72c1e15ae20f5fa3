"""torch.autograd wrapper of the converged RIC-MRCCSD energy.

`RicMrccEnergy.apply(h, B, s, handle, opts)` sets the integrals on a handle
whose RDMs are already set, solves (Eq. ric-update) and returns E; backward
returns dE/dh, dE/dB, dE/ds from the library's hand-written adjoint
(`ricmrcc_energy_backward`).  The orbital basis is held fixed.
"""
from __future__ import annotations

import numpy as np
import torch


class RicMrccEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, B, s, handle, opts=None):
        opts = dict(opts or {})
        handle.set_integrals(np.ascontiguousarray(h.detach().cpu().numpy()),
                             np.ascontiguousarray(B.detach().cpu().numpy()))
        e, st = handle.solve(float(s), **opts)
        if st.converged != 1:
            raise RuntimeError("RIC-MRCCSD solve did not converge")
        ctx.handle = handle
        ctx.like = (h, B, s)
        return torch.tensor(e, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, g):
        dh, dB, ds = ctx.handle.energy_backward()
        h, B, s = ctx.like
        gh = g * torch.tensor(dh, dtype=h.dtype, device=h.device)
        gB = g * torch.tensor(dB, dtype=B.dtype, device=B.device)
        gs = g * torch.tensor(ds, dtype=torch.float64, device=h.device) if torch.is_tensor(s) else None
        return gh, gB, gs, None, None
