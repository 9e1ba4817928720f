"""torch.autograd.Function wrappers of the CUDA forward and adjoint entry points.

    psi_T = anneal(psi0, h, J, gammas, ts)        # differentiable in all five
    L = energy(psi_T, h, J)                       # <psi|H_P|psi>, differentiable
    L.backward()

psi0 and psi_T are CUDA complex tensors (complex64 or complex128); h (n), J (n x n,
upper triangle used), gammas (S) and ts (S) are float64 tensors on any device.
Forward and backward both run in the CUDA library (cheb_anneal,
cheb_anneal_adjoint, cheb_energy_grad); this module only moves arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def _np(x):
    return x.detach().to("cpu", torch.float64).numpy()


class AnnealFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, h, J, gammas, ts, tol, method, store_vectors):
        hn, Jn, gn, tn = _np(h), _np(J), _np(gammas), _np(ts)
        S = gn.shape[0]
        y = psi0.detach().clone().contiguous()
        bnd = torch.empty((S, y.numel()), dtype=y.dtype, device=y.device)
        api.anneal(hn, Jn, gn, tn, y, tol=tol, method=method, boundaries=bnd, info=False)
        ctx.save_for_backward(bnd, y)
        ctx.params = (hn, Jn, gn, tn, tol, method, store_vectors)
        ctx.dev = (h.device, J.device, gammas.device, ts.device)
        return y

    @staticmethod
    def backward(ctx, grad_out):
        bnd, y = ctx.saved_tensors
        hn, Jn, gn, tn, tol, method, store_vectors = ctx.params
        g = grad_out.detach().to(y.dtype).contiguous().clone()
        out = api.anneal_adjoint(hn, Jn, gn, tn, bnd, y, g, tol=tol, method=method, store_vectors=store_vectors)
        dh = torch.from_numpy(out["h"]).to(ctx.dev[0])
        dJ = torch.from_numpy(out["J"]).to(ctx.dev[1])
        dg = torch.from_numpy(out["gamma"]).to(ctx.dev[2])
        dt = torch.from_numpy(out["t"]).to(ctx.dev[3])
        return g, dh, dJ, dg, dt, None, None, None


class EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, h, J):
        e, g, gh, gJ = api.energy_grad(_np(h), _np(J), psi.detach().contiguous())
        ctx.save_for_backward(g)
        ctx.grads = (torch.from_numpy(gh).to(h.device), torch.from_numpy(gJ).to(J.device))
        return torch.tensor(e, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        gh, gJ = ctx.grads
        s = float(grad_out)
        return g * s, gh * s, gJ * s


def anneal(psi0, h, J, gammas, ts, tol=None, method="chebyshev", store_vectors=None):
    return AnnealFn.apply(psi0, h, J, gammas, ts, tol, method, store_vectors)


def expmv(psi0, h, J, gamma, t, tol=None, method="chebyshev", store_vectors=None):
    """Differentiable exp(-i t H) psi0 (a one-segment schedule)."""
    g = gamma.reshape(1) if isinstance(gamma, torch.Tensor) else torch.tensor([float(gamma)], dtype=torch.float64)
    tt = t.reshape(1) if isinstance(t, torch.Tensor) else torch.tensor([float(t)], dtype=torch.float64)
    return AnnealFn.apply(psi0, h, J, g, tt, tol, method, store_vectors)


def energy(psi, h, J):
    return EnergyFn.apply(psi, h, J)
