"""Variance tuning of the per-graph densities (the adjoint path).

`SecondMoment` is a torch.autograd.Function whose forward returns the Monte
Carlo estimate of M2(theta) = E_p[(f/p)^2] for a loaded graph and whose
backward returns dM2/dtheta from the library's adjoint kernel (points are
recomputed from their Philox counters, never stored).  theta = (alpha, beta):
per-line shifts of Deg and first-step sector weights.  Any theta keeps the
estimator unbiased; lowering M2 lowers its variance.  torch only holds the
parameters and runs the optimiser; every sample is evaluated by the library.
"""
from __future__ import annotations

import ctypes as C

import torch

from ._lib import _check, load_library


def _set_params(diag, alpha, beta):
    N = diag.n_lines
    a = (C.c_double * N)(*[float(x) for x in alpha])
    b = (C.c_double * N)(*[float(x) for x in beta])
    _check(load_library().qed_diagram_set_pdf_params(diag._h, a, b))


def pdf_grad(diag, alpha, beta, n, seed=0, begin=0):
    """(M2, dM2/dalpha, dM2/dbeta) at theta = (alpha, beta)."""
    L = load_library()
    if not hasattr(L.qed_pdf_grad, "_typed"):
        L.qed_pdf_grad.restype = C.c_int
        L.qed_pdf_grad.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.qed_diagram_set_pdf_params.restype = C.c_int
        L.qed_diagram_set_pdf_params.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.qed_pdf_grad._typed = True
    _set_params(diag, alpha, beta)
    N = diag.n_lines
    m2 = C.c_double()
    g = (C.c_double * (2 * N))()
    _check(L.qed_pdf_grad(diag._h, begin, n, seed, C.byref(m2), g))
    return m2.value, list(g[:N]), list(g[N:])


class SecondMoment(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, beta, diag, n, seed, begin):
        m2, ga, gb = pdf_grad(diag, alpha.detach().cpu().tolist(), beta.detach().cpu().tolist(), n, seed, begin)
        ctx.save_for_backward(torch.tensor(ga, dtype=alpha.dtype), torch.tensor(gb, dtype=beta.dtype))
        return torch.tensor(m2, dtype=alpha.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        ga, gb = ctx.saved_tensors
        return grad_out * ga, grad_out * gb, None, None, None, None


def tune(diag, steps=20, n=1 << 22, lr=0.05, seed=1234, log=None):
    """Adam on theta to lower M2; fresh counters every step (unbiased
    gradient estimates).  Leaves the best theta seen loaded in the graph and
    returns (alpha, beta, history of M2)."""
    N = diag.n_lines
    alpha = torch.zeros(N, dtype=torch.float64, requires_grad=True)
    beta = torch.zeros(N, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([alpha, beta], lr=lr)
    hist = []
    best = (float("inf"), None, None)
    for s in range(steps):
        opt.zero_grad()
        m2 = SecondMoment.apply(alpha, beta, diag, n, seed, (s + 1) * n)
        m2.backward()
        hist.append(m2.item())
        if m2.item() < best[0]:
            best = (m2.item(), alpha.detach().clone(), beta.detach().clone())
        opt.step()
        with torch.no_grad():
            alpha.clamp_(-0.45, 2.0)
            beta.clamp_(-3.0, 3.0)
        if log:
            log(s, m2.item())
    _set_params(diag, best[1].tolist(), best[2].tolist())
    return best[1], best[2], hist
