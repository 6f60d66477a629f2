"""Differentiable 2F and gradient-ascent refinement of candidates.

``TwoF`` is a torch.autograd.Function over fstat_grad: the forward pass
evaluates 2F at theta = (f, f1dot, alpha, delta) (float64, one row per
candidate) with the demodulation sums of eqs. (Fa_DET)/(Fb_DET) of Sec. 2;
the backward pass multiplies the incoming gradient by the adjoint's
d2F/dtheta.  ``refine`` runs gradient ascent with per-candidate step
control, the whole loop on the device (fstat_refine).
"""

from __future__ import annotations

import numpy as np
import torch

from . import CANDIDATE_DTYPE


def _candidates(theta: torch.Tensor, f2dot) -> np.ndarray:
    t = theta.detach().to("cpu", torch.float64).numpy()
    c = np.empty(len(t), dtype=CANDIDATE_DTYPE)
    c["f"], c["f1dot"], c["alpha"], c["delta"] = t[:, 0], t[:, 1], t[:, 2], t[:, 3]
    c["f2dot"] = np.broadcast_to(np.asarray(f2dot, dtype=np.float64), (len(t),))
    return c


class TwoF(torch.autograd.Function):
    """2F(theta) with d2F/dtheta from the hand-written adjoint kernel."""

    @staticmethod
    def forward(ctx, theta, plan, f2dot=0.0):
        two_f, g = plan.grad(_candidates(theta, f2dot))
        ctx.save_for_backward(g)
        ctx.theta_meta = (theta.dtype, theta.device)
        return two_f.to(theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        dtype, device = ctx.theta_meta
        gt = g.to(device=device, dtype=dtype) * grad_out.to(device=device, dtype=dtype)[:, None]
        return gt, None, None


def twoF(theta: torch.Tensor, plan, f2dot=0.0) -> torch.Tensor:
    return TwoF.apply(theta, plan, f2dot)


def refine(plan, theta0, scales, steps: int = 20, f2dot=0.0, step0: float = 0.25):
    """Gradient ascent on 2F from theta0 ([n, 4], float64).

    ``scales`` ([4]) are the natural spacings of (f, f1dot, alpha, delta);
    the step moves ``eta`` scaled units along the scaled gradient direction,
    with eta growing by 1.25 on accepted steps and halving on rejected ones
    (a step that lowers 2F is not taken).  The loop runs on the device
    (fstat_refine).  Returns (theta [n, 4] float64, 2F history [steps+1, n]
    float64)."""
    theta = torch.as_tensor(theta0, dtype=torch.float64)
    out, hist = plan.refine(_candidates(theta, f2dot), np.asarray(scales, dtype=np.float64), steps=steps,
                            step0=step0)
    th = np.stack([out["f"], out["f1dot"], out["alpha"], out["delta"]], axis=1)
    return torch.from_numpy(th), torch.from_numpy(hist.astype(np.float64))
