"""``torch.autograd.Function`` over the library's gradient entry points.

``MicrocircuitRates.apply(scales, nu, net, n_steps, ckpt_every, start_state)``
returns the population rates (Hz) of ``n_steps`` steps of ``net`` run with
projection weight scales ``scales`` [8][8] (target, source) and background
rate ``nu`` (Hz), starting from ``start_state`` (bytes from
``Microcircuit.save_state``; None continues from the current state).  Its
backward is ``snn_grad_backward``: surrogate-gradient backpropagation through
time on the device.  Argument marshalling only.
"""
from __future__ import annotations

import numpy as np
import torch


class MicrocircuitRates(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scales, nu, net, n_steps, ckpt_every=100, start_state=None):
        if start_state is not None:
            net.load_state(start_state)
        net.set_params(scales.detach().to("cpu", torch.float64).numpy(), float(nu))
        rates = net.grad_forward(int(n_steps), int(ckpt_every))
        ctx.net = net
        ctx.meta = (scales.dtype, scales.device, nu.dtype, nu.device)
        return torch.as_tensor(rates, dtype=torch.float64, device=scales.device)

    @staticmethod
    def backward(ctx, grad_rates):
        ga, gn = ctx.net.grad_backward(grad_rates.detach().to("cpu", torch.float64).numpy())
        sd, sdev, nd, ndev = ctx.meta
        g_scales = torch.as_tensor(np.ascontiguousarray(ga), dtype=sd, device=sdev)
        g_nu = torch.as_tensor(gn, dtype=nd, device=ndev)
        return g_scales, g_nu, None, None, None, None


def microcircuit_rates(scales, nu, net, n_steps, ckpt_every=100, start_state=None):
    return MicrocircuitRates.apply(scales, nu, net, n_steps, ckpt_every, start_state)
