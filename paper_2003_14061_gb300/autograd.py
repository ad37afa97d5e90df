"""torch.autograd.Function over the library's trajectory adjoint (md_adjoint).

    loss = MDTrajectoryFn.apply(eps, sigma, v0, x0, box, nsteps, ckpt_every, options)

eps and sigma are scalar tensors, v0 a float64 [n, 3] tensor (the initial velocities), x0 and box
the initial positions and box (not differentiated).  The loss is
L = (1/S) sum_{n=1..S} U(x_n) + |v_S|^2 over S = nsteps leapfrog steps.  The forward call runs the
trajectory and its reverse pass together (one md_adjoint call), and backward scales the stored
gradients by the incoming gradient.  With the WCA cutoff (options["rc_over_sigma"] = 2^(1/6),
the default) the cutoff moves with sigma.
"""
from __future__ import annotations

import numpy as np
import torch

from .system import MDSystem

WCA_RC_OVER_SIGMA = 2.0 ** (1.0 / 6.0)


class MDTrajectoryFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, sigma, v0, x0, box, nsteps, ckpt_every=20, options=None):
        opts = dict(options or {})
        rc_over_sigma = opts.pop("rc_over_sigma", WCA_RC_OVER_SIGMA)
        device = opts.pop("device", None)
        e = float(eps.detach().cpu())
        s = float(sigma.detach().cpu())
        opts.setdefault("precision", "mixed")
        opts.setdefault("skin", 0.4)
        x0_np = x0.detach().cpu().numpy() if isinstance(x0, torch.Tensor) else np.asarray(x0, dtype=np.float64)
        box_np = box.detach().cpu().numpy() if isinstance(box, torch.Tensor) else np.asarray(box, dtype=np.float64)
        v0_np = v0.detach().to(torch.float64).cpu().numpy()
        sysm = MDSystem(x0_np, v0_np, box_np, eps=e, sigma=s, rc=rc_over_sigma * s, device=device, **opts)
        try:
            loss, ge, gs, gv = sysm.adjoint(int(nsteps), int(ckpt_every))
        finally:
            sysm.close()
        ctx.save_for_backward(torch.tensor(ge, dtype=torch.float64), torch.tensor(gs, dtype=torch.float64),
                              torch.from_numpy(gv))
        ctx.v0_device = v0.device
        ctx.v0_dtype = v0.dtype
        return torch.tensor(loss, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        ge, gs, gv = ctx.saved_tensors
        go = grad_out.detach().to(torch.float64).cpu()
        d_eps = (go * ge).to(grad_out.device)
        d_sig = (go * gs).to(grad_out.device)
        d_v0 = (go * gv).to(device=ctx.v0_device, dtype=ctx.v0_dtype)
        return d_eps, d_sig, d_v0, None, None, None, None, None
