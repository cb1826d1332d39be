"""chi^2 of the fused RIME as a differentiable torch function.

``RimeChi2.apply(rime, lm, stokes, alpha, shape, gains)`` uploads the sky
model (and gains, if given) to the context, evaluates chi^2 and its adjoint
with ``rime_chi2_grad`` in one pass, and returns chi^2 as a 0-d float64
tensor; backward scales the stored gradients by the incoming gradient. All
parameters are float64 (gains complex128) tensors; the gradient of the gains
follows torch's convention for complex inputs (d/dRe + i d/dIm).
"""
import torch


class RimeChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rime, lm, stokes, alpha, shape, gains=None):
        src = dict(lm=lm.detach().contiguous(), stokes=stokes.detach().contiguous(),
                   alpha=alpha.detach().contiguous(),
                   shape=None if shape is None else shape.detach().contiguous())
        rime.set_sources(src)
        if gains is not None:
            rime.set_gains(gains.detach().contiguous())
        chi, gs, gg = rime.chi2_grad(want_gains=gains is not None)
        ctx.save_for_backward(gs)
        ctx.gg = gg
        ctx.has_shape = shape is not None
        return torch.tensor(chi, dtype=torch.float64, device=lm.device)

    @staticmethod
    def backward(ctx, grad_out):
        (gs,) = ctx.saved_tensors
        g = grad_out.to(gs.device)
        d_lm = g * gs[:, 0:2]
        d_stokes = g * gs[:, 2:6]
        d_alpha = g * gs[:, 6]
        d_shape = g * gs[:, 7:10] if ctx.has_shape else None
        d_gains = None
        if ctx.gg is not None:
            d_gains = g.to(torch.complex128) * ctx.gg
        return None, d_lm, d_stokes, d_alpha, d_shape, d_gains
