"""Oracle adjoint (test infrastructure only): gradients of Re<ubar, u> with
respect to the boundary data g, the source f and the coefficient c, written
from the dense composite collocation system of oracle.composite, with no
merge recursion.

The discrete solution solves A(c) s = rhs(f, g) and u = E s + u_g(g) (DtN:
interior values from s, boundary nodes from the interface unknowns and g;
ItI: u = s).  For J = Re<ubar, u>:
    lambda = A^{-H} E^H ubar,
    dJ/df at the leaf interior nodes = the entries of lambda on the rows
        where f enters (the leaf interior equations),
    dJ/dg = M^H ubar with M the (exactly linear) map g -> u at f = 0, formed
        column by column from unit vectors (brute force),
    dJ/dc_j = -Re(conj(lambda_row(j)) u_j) at interior node j, because c
        enters A only on the diagonal of the leaf interior equations
        (L = a Lap + b.grad + c, Section 2).
Pins (tests/test_oracle_adjoint.py): central finite differences of J in c,
and the identity Re<ubar, u(g, f)> = Re<gbar, g> + Re<fbar, f>.
"""

from __future__ import annotations

import numpy as np

from . import composite as O2
from . import leaf as lf


def adjoint_dtn(dim, p, L, lo, hi, a, b, c, f, g, ubar, with_gbar=True):
    """(gbar, fbar, grad_c, u) for the DtN composite system (gbar None when
    with_gbar is False: it takes one dense solve per boundary value)."""
    A, rhs, unpack = O2.assemble_dtn(dim, p, L, lo, hi, a, b, c, f, g)
    info = unpack.info
    nl, npts, ni, npan, off_g = info["nl"], info["npts"], info["ni"], info["npan"], info["off_g"]
    Ie, Ii, P = info["Ie"], info["Ii"], info["P"]
    sol = np.linalg.solve(A, rhs)
    u = unpack(sol, g)
    # E^H ubar: interior values and the interface-panel part of P g_leaf
    sbar = np.zeros(A.shape[0], np.result_type(ubar, sol))
    for m in range(nl):
        sbar[m * ni:(m + 1) * ni] += ubar[m, Ii]
        pb = P.T @ ubar[m, Ie]
        for s, (kind, k) in enumerate(info["panels"][m]):
            if kind == "int":
                sbar[off_g + k * npan:off_g + (k + 1) * npan] += pb[s * npan:(s + 1) * npan]
    lam = np.linalg.solve(A.conj().T, sbar)
    fbar = np.zeros((nl, npts), lam.dtype)
    grad_c = np.zeros((nl, npts))
    for m in range(nl):
        fbar[m, Ii] = lam[m * ni:(m + 1) * ni]
        grad_c[m, Ii] = -np.real(np.conj(lam[m * ni:(m + 1) * ni]) * u[m, Ii])
    gbar = None
    if with_gbar:
        gbar = _gbar_by_columns(lambda gg: O2.solve_dtn(dim, p, L, lo, hi, a, b, c, np.zeros_like(f), gg),
                                g, ubar)
    return gbar, fbar, grad_c, u


def adjoint_iti(p, L, lo, hi, a, b, c, f, g, ubar, eta):
    """(gbar, fbar, grad_c, u) for the ItI composite system."""
    A, rhs = O2.assemble_iti(p, L, lo, hi, a, b, c, f, g, eta)
    nl, npl = (2 ** L) ** 2, p * p
    ops = lf.reference_ops(2, p, p - 2)
    Ii = ops["Ii"]
    nown = lf.iti_ops(p, p - 2, 1.0, eta)[1].shape[0]
    sol = np.linalg.solve(A, rhs)
    u = sol.reshape(nl, npl)
    lam = np.linalg.solve(A.conj().T, ubar.reshape(-1)).reshape(nl, npl)
    fbar = np.zeros((nl, npl), complex)
    grad_c = np.zeros((nl, npl))
    for m in range(nl):
        lint = lam[m, nown:nown + len(Ii)]
        fbar[m, Ii] = lint
        grad_c[m, Ii] = -np.real(np.conj(lint) * u[m, Ii])
    gbar = _gbar_by_columns(lambda gg: O2.solve_iti(p, L, lo, hi, a, b, c, np.zeros_like(f), gg, eta), g, ubar)
    return gbar, fbar, grad_c, u


def _gbar_by_columns(solve_g, g, ubar):
    """M^H ubar for the linear map g -> u (f = 0), one column per unit vector."""
    gbar = np.zeros(g.shape, np.result_type(g, ubar, complex) if np.iscomplexobj(g) or np.iscomplexobj(ubar)
                    else float)
    for i in range(g.size):
        e = np.zeros_like(g)
        e.flat[i] = 1.0
        gbar.flat[i] = np.vdot(solve_g(e), ubar)
    return gbar
