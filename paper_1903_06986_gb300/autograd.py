"""torch.autograd interface to the scalar loop estimate (Sec. 5-6): Re of the unsubtracted noise
estimate of Tr M^{-1} as a differentiable function of kappa and of the gauge links.

The forward pass calls lqcd_loop_estimate; the backward pass calls lqcd_loop_derivs, which re-solves
the systems it needs (x = M^{-1} eta, y = M^{-1} P x and the adjoint M^{-dag} eta) instead of keeping
Krylov bases from the forward pass, and returns d/dkappa and the gradient with respect to the
complex link entries in torch's convention (dT/dU* + conj(dT/dU) for the real output).  The
upstream gradient is passed to the library as its scale; this module only marshals arguments.
"""
import torch

from . import lqcd


class ScalarLoopEstimate(torch.autograd.Function):
    """f(kappa, links) = Re (1/N) sum_n eta_n^dag M(kappa, links)^{-1} eta_n for the Z(4) noises of
    opts['seed']; opts holds the solver settings of Context.loop_estimate (nnoise, block, m, k, K,
    npoly, tol, tol_special, and optionally m_inner, max_cycles, prec)."""

    @staticmethod
    def forward(fctx, kappa, links, lctx, opts):
        r = lctx.loop_estimate(links, float(kappa), modes=lqcd.SUB_NONE, **opts)
        fctx.save_for_backward(kappa, links)
        fctx.lctx = lctx
        fctx.opts = opts
        return torch.tensor(r["mean"][0, 0].real, dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        kappa, links = fctx.saved_tensors
        o = fctx.opts
        g = float(grad_out)
        d = lqcd.loop_derivs(fctx.lctx, links, float(kappa), o["seed"], o["nnoise"], o["block"], o["m"], o["k"],
                             o["K"], o["tol"], o["tol_special"], m_inner=o.get("m_inner", 0),
                             max_cycles=o.get("max_cycles", 2000), prec=o.get("prec", lqcd.PREC_F64),
                             want_grad=bool(fctx.needs_input_grad[1]), grad_scale=g)
        gk = torch.tensor(d["dkappa"][0, 0].real * g, dtype=kappa.dtype, device=kappa.device)
        return gk, d["grad_links"], None, None


def scalar_loop(kappa, links, lctx, **opts):
    """Differentiable Re (noise estimate of Tr M^{-1}); kappa: 0-d float64 tensor, links: complex128."""
    return ScalarLoopEstimate.apply(kappa, links, lctx, opts)
