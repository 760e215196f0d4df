"""torch.autograd wrapper: cross sections as a differentiable function of model parameters.

Forward: build the model with the given parameter values, solve every (eps_i, v_i, mu)
system (Eq. Ax=b) and form sigma (Eq. crs).  The solutions psi are kept (one checkpoint
per energy) for the backward pass, which calls the library's adjoint solve with the same
complex-symmetric operator.  Parameter ids follow ``vbk_solve_adjoint``: k < n_terms is the
coefficient of term k, n_terms + 2c / n_terms + 2c + 1 are a / b of channel c, and
n_terms + 2 n_channels + t is the coefficient of coupling-polynomial term t, counted channel by
channel in listed order (the order in which the binding passes them to the library).
"""

from __future__ import annotations

import copy

import torch


def _with_values(desc: dict, theta_ids, values) -> dict:
    m = copy.deepcopy(desc)
    nt, nc = len(m["terms"]), len(m["channels"])
    cterms = [t for c in m["channels"] for t in (c.get("terms") or [])]
    for tid, v in zip(theta_ids, values):
        tid = int(tid)
        if tid < nt:
            m["terms"][tid]["coef"] = float(v)
        elif tid < nt + 2 * nc:
            c, which = divmod(tid - nt, 2)
            m["channels"][c]["ab"[which]] = float(v)
        else:
            cterms[tid - nt - 2 * nc]["coef"] = float(v)
    return m


class CrossSectionFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, desc, theta_ids, eps, vi, vf, opts):
        from . import Model, vbk_cross_sections, vbk_solve

        model = Model(_with_values(desc, theta_ids, theta.detach().cpu().tolist()))
        psi, stats = vbk_solve(model, eps, vi, opts)
        sigma = vbk_cross_sections(model, eps, vi, psi, vf)
        ctx.model, ctx.psi = model, psi
        ctx.args = (theta_ids, eps, vi, vf, opts)
        ctx.stats = stats
        return sigma

    @staticmethod
    def backward(ctx, grad_sigma):
        from . import vbk_solve_adjoint

        theta_ids, eps, vi, vf, opts = ctx.args
        grad, _ = vbk_solve_adjoint(ctx.model, eps, vi, ctx.psi, vf, grad_sigma.to(torch.float64).contiguous(),
                                    theta_ids, opts)
        g = torch.as_tensor(grad, dtype=torch.float64)
        return g, None, None, None, None, None, None


def cross_sections_torch(theta, desc, theta_ids, eps, vi, vf, opts=None):
    """sigma[e, i, f] as a differentiable function of ``theta`` (float64 tensor)."""
    return CrossSectionFunction.apply(theta, desc, list(theta_ids), eps, vi, vf, opts)
