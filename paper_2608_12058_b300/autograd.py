"""torch.autograd.Function wrappers of the CUDA forward and adjoint entry points.

    psi_T = anneal(psi0, h, J, gammas, ts)        # differentiable in all five
    psi_T = anneal_general(psi0, h, J, a_s, b_s, ts)    # segments b_s H_P + a_s sum X_j
    psi_T = magnus4(psi0, h, J, dt, nodes)        # time-dependent H(t), Magnus steps
    L = energy(psi_T, h, J)                       # <psi|H_P|psi>, differentiable
    L.backward()

psi0 and psi_T are CUDA complex tensors (complex64 or complex128); h (n), J (n x n,
upper triangle used), gammas (S) and ts (S) are float64 tensors on any device.
Forward and backward both run in the CUDA library (cheb_anneal, cheb_magnus4,
cheb_anneal_adjoint, cheb_magnus4_adjoint, cheb_energy_grad); this module only
moves arguments.
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
        ctx.ckpt = None
        if any(ctx.needs_input_grad[:5]):
            # the adjoint then skips the last segment's forward recomputation
            ctx.ckpt = api.anneal_checkpointed(hn, Jn, gn, tn, y, bnd, tol=tol, method=method,
                                               store_vectors=store_vectors)
        else:
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
        out = api.anneal_adjoint(hn, Jn, gn, tn, bnd, y, g, tol=tol, method=method, store_vectors=store_vectors,
                                 checkpoint=ctx.ckpt)
        ctx.ckpt = None
        dh = torch.from_numpy(out["h"]).to(ctx.dev[0])
        dJ = torch.from_numpy(out["J"]).to(ctx.dev[1])
        dg = torch.from_numpy(out["gamma"]).to(ctx.dev[2])
        dt = torch.from_numpy(out["t"]).to(ctx.dev[3])
        return g, dh, dJ, dg, dt, None, None, None


class AnnealGeneralFn(torch.autograd.Function):
    """psi_T = prod_s exp(-i t_s (b_s H_P + a_s sum_j X_j)) psi0, differentiable in psi0, h,
    J, a_s, b_s and t_s (cheb_anneal_general / cheb_anneal_general_adjoint)."""

    @staticmethod
    def forward(ctx, psi0, h, J, a_s, b_s, ts, tol, method, store_vectors):
        hn, Jn, an, bn, tn = _np(h), _np(J), _np(a_s), _np(b_s), _np(ts)
        S = an.shape[0]
        y = psi0.detach().clone().contiguous()
        bnd = torch.empty((S, y.numel()), dtype=y.dtype, device=y.device)
        ctx.ckpt = None
        if any(ctx.needs_input_grad[:6]):
            ctx.ckpt = api.anneal_general_checkpointed(hn, Jn, an, bn, tn, y, bnd, tol=tol, method=method,
                                                       store_vectors=store_vectors)
        else:
            api.anneal_general(hn, Jn, an, bn, tn, y, tol=tol, method=method, boundaries=bnd, info=False)
        ctx.save_for_backward(bnd, y)
        ctx.params = (hn, Jn, an, bn, tn, tol, method, store_vectors)
        ctx.dev = (h.device, J.device, a_s.device, b_s.device, ts.device)
        return y

    @staticmethod
    def backward(ctx, grad_out):
        bnd, y = ctx.saved_tensors
        hn, Jn, an, bn, tn, tol, method, store_vectors = ctx.params
        g = grad_out.detach().to(y.dtype).contiguous().clone()
        out = api.anneal_general_adjoint(hn, Jn, an, bn, tn, bnd, y, g, tol=tol, method=method,
                                         store_vectors=store_vectors, checkpoint=ctx.ckpt)
        ctx.ckpt = None
        conv = lambda key, dev: torch.from_numpy(out[key]).to(dev)
        return (g, conv("h", ctx.dev[0]), conv("J", ctx.dev[1]), conv("a", ctx.dev[2]), conv("b", ctx.dev[3]),
                conv("t", ctx.dev[4]), None, None, None)


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


def anneal_general(psi0, h, J, a_s, b_s, ts, tol=None, method="chebyshev", store_vectors=None):
    return AnnealGeneralFn.apply(psi0, h, J, a_s, b_s, ts, tol, method, store_vectors)


class Magnus4Fn(torch.autograd.Function):
    """psi_T = the fourth-order Magnus propagator of H(t) = A(t) sum_j X_j + B(t) H_P applied
    to psi0 (cheb_magnus4), differentiable in psi0, h, J, the step lengths dt and the node
    values (cheb_magnus4_adjoint)."""

    @staticmethod
    def forward(ctx, psi0, h, J, dt, nodes, tol, method, store_vectors):
        hn, Jn, dn, nn = _np(h), _np(J), _np(dt), _np(nodes)
        steps = dn.shape[0]
        y = psi0.detach().clone().contiguous()
        bnd = torch.empty((2 * steps, y.numel()), dtype=y.dtype, device=y.device)
        api.magnus4(hn, Jn, dn, nn, y, tol=tol, method=method, boundaries=bnd)
        ctx.save_for_backward(bnd, y)
        ctx.params = (hn, Jn, dn, nn, tol, method, store_vectors)
        ctx.dev = (h.device, J.device, dt.device, nodes.device)
        ctx.nshape = tuple(nodes.shape)
        return y

    @staticmethod
    def backward(ctx, grad_out):
        bnd, y = ctx.saved_tensors
        hn, Jn, dn, nn, tol, method, store_vectors = ctx.params
        g = grad_out.detach().to(y.dtype).contiguous().clone()
        out = api.magnus4_adjoint(hn, Jn, dn, nn, bnd, y, g, tol=tol, method=method, store_vectors=store_vectors)
        conv = lambda key, dev: torch.from_numpy(out[key]).to(dev)
        return (g, conv("h", ctx.dev[0]), conv("J", ctx.dev[1]), conv("dt", ctx.dev[2]),
                conv("nodes", ctx.dev[3]).reshape(ctx.nshape), None, None, None)


def magnus4(psi0, h, J, dt, nodes, tol=None, method="chebyshev", store_vectors=None):
    """Differentiable fourth-order commutator-free Magnus propagation (as api.magnus4):
    dt (steps) and nodes (steps x 4: A(t1), B(t1), A(t2), B(t2)) are float64 tensors;
    gradients reach dt and every node value through cheb_magnus4_adjoint."""
    return Magnus4Fn.apply(psi0, h, J, dt, nodes, tol, method, store_vectors)


def energy(psi, h, J):
    return EnergyFn.apply(psi, h, J)
