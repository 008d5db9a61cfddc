"""Differentiation through T-REXI steps.

``RexiStep`` is a ``torch.autograd.Function`` whose backward is the library's
hand-written adjoint step (``rexi_step_adjoint``: the transposed transforms and
sum_k conj(beta_k) (conj(alpha_k) + tau L^H)^{-1}), so dJ/dU0 of any scalar misfit
J(U(T)) flows through a rollout of REXI steps.  The step is linear, so its
backward needs none of the forward states; ``rollout`` still accepts a
checkpoint interval so that rollouts mixed with other (nonlinear) torch
operations recompute segments instead of storing them.
"""
import torch
from torch.utils.checkpoint import checkpoint


class RexiStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.step(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.step_adjoint(g.contiguous()), None


def rexi_step(plan, x):
    """One differentiable T-REXI step of ``plan`` applied to x (layout of the plan)."""
    return RexiStep.apply(x, plan)


def rollout(plan, x0, nsteps, checkpoint_every=0, extra=None):
    """U(n tau) after ``nsteps`` differentiable steps.

    ``extra`` (optional callable) is applied after every step (e.g. a forcing or a
    nonlinear correction).  With ``checkpoint_every = k > 0`` the rollout is split
    into segments of k steps wrapped in ``torch.utils.checkpoint`` (non-reentrant),
    which store only segment inputs and recompute the rest in the backward pass.
    """
    def segment(x, k):
        for _ in range(k):
            x = RexiStep.apply(x, plan)
            if extra is not None:
                x = extra(x)
        return x

    x = x0
    done = 0
    while done < nsteps:
        k = nsteps - done if checkpoint_every <= 0 else min(checkpoint_every, nsteps - done)
        if checkpoint_every > 0 and torch.is_grad_enabled():
            x = checkpoint(segment, x, k, use_reentrant=False)
        else:
            x = segment(x, k)
        done += k
    return x
