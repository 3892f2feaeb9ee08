"""torch.autograd.Function over ptsbe_backward: the fixed-set estimator of a diagonal observable
as a differentiable function of the gate angles and channel strengths.

The Kraus sets (and their nominal probabilities and multiplicities) are drawn once and held fixed;
each forward registers the circuit at the given parameters and runs the library's adjoint kernels,
which return the loss and its full gradient together; backward scales that gradient by the
incoming one. Argument marshalling only: every step runs in libptsbe.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch


class FixedSetLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op_params, ch_params, runtime, circ, info, first, count, masks, coeffs, diag, checkpoint_every):
        c2 = dataclasses.replace(circ, op_params=op_params.detach().cpu().numpy().astype(np.float64).reshape(-1, 3),
                                 ch_params=ch_params.detach().cpu().numpy().astype(np.float64).reshape(-1))
        dev = torch.device("cuda", runtime.device)
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        gp = torch.empty((circ.n_ops, 3), dtype=torch.float64, device=dev)
        gn = torch.empty(max(len(circ.ch_params), 1), dtype=torch.float64, device=dev)
        cid = runtime.register(c2)
        try:
            runtime.backward(cid, info, first, count, masks, coeffs, diag=diag, checkpoint_every=checkpoint_every,
                             loss=loss, grad_params=gp, grad_noise=gn)
            runtime.synchronize()
        finally:
            runtime.release_circuit(cid)
        ctx.save_for_backward(gp.to(op_params.device, op_params.dtype),
                              gn[: len(circ.ch_params)].to(ch_params.device, ch_params.dtype))
        return loss[0].to(op_params.device, op_params.dtype)

    @staticmethod
    def backward(ctx, g):
        gp, gn = ctx.saved_tensors
        return g * gp, g * gn, None, None, None, None, None, None, None, None, None


def fixed_set_loss(op_params, ch_params, runtime, circ, info, first=0, count=None, masks=(), coeffs=(), diag=None,
                   checkpoint_every=0):
    """L(op_params [n_ops, 3], ch_params [n_channels]) with gradients through ptsbe_backward."""
    if count is None:
        count = info.count - first
    return FixedSetLoss.apply(op_params, ch_params, runtime, circ, info, first, count, masks, coeffs, diag,
                              checkpoint_every)
