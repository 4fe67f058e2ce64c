"""torch.autograd.Function over the C ABI: u = HPS solve for the coefficient
field c (at the leaf nodes), root boundary data g and source f, with a
backward pass that runs the library's adjoint solve (hps_solve_adjoint) and
coefficient-gradient kernel (hps_coeff_gradient) on the stored factors.

Gradients follow PyTorch's convention for complex tensors (the conjugate
Wirtinger derivative): for u = A_g g + A_f f the backward returns
grad_g = A_g^H grad_u and grad_f = A_f^H grad_u, and for the real c,
grad_c = -Re(conj(A_f^H grad_u) u) at the leaf interior nodes (zero at leaf
boundary nodes, whose equations do not involve the coefficients).
"""

from __future__ import annotations

import torch

from . import (HPS_DTN, HPS_ITI, hps_build, hps_coeff_gradient, hps_free, hps_solve,  # noqa: F401
               hps_solve_adjoint)


class HPSSolve(torch.autograd.Function):
    """u = HPSSolve.apply(c, g, f, tree, p, kind, a, b, eta, lazy_root).

    c: float64 [n_leaves, p^d] (device), g: [n_root_bdry], f: [n_leaves, p^d]
    (float64 for DtN, complex128 for ItI); a and b: fixed coefficient arrays
    (or None for a = 1, b = 0).  The handle built in forward stays on the
    autograd context, so every backward through the graph (retain_graph=True,
    or torch.autograd.grad called more than once) reuses its factors; it is
    released when the graph is freed (Handle.__del__ calls hps_free)."""

    @staticmethod
    def forward(ctx, c, g, f, tree, p, kind, a=None, b=None, eta=0.0, lazy_root=False):
        c, g, f = c.contiguous(), g.contiguous(), f.contiguous()
        h = hps_build(tree, p, p - 2, kind, a=a, b=b, c=c, f=f, eta=eta, lazy_root=lazy_root)
        u = torch.empty_like(f)
        hps_solve(h, g, u)
        ctx.h = h
        ctx.g_shape = g.shape
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        h = ctx.h
        gbar = torch.empty(ctx.g_shape, dtype=u.dtype, device=u.device)
        fbar = torch.empty_like(u)
        hps_solve_adjoint(h, grad_u.contiguous(), gbar, fbar)
        gc = torch.empty(u.shape, dtype=torch.float64, device=u.device)
        hps_coeff_gradient(h, u, fbar, gc=gc)
        return gc, gbar, fbar, None, None, None, None, None, None, None


def hps_solve_fn(c, g, f, tree, p, kind, a=None, b=None, eta=0.0, lazy_root=False):
    """Functional form of HPSSolve.apply."""
    return HPSSolve.apply(c, g, f, tree, p, kind, a, b, eta, lazy_root)
