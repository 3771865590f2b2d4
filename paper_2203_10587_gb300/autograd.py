"""torch.autograd.Function wrappers over the C ABI's evaluation and adjoint kernels.

The constraint map c(x) = [g(x); h(x)] (ExaGO, Sec. III, eqs. (8)-(9)) and the objective f(x)
(eq. (7), weighted by pi_s for scenarios, eq. (27)) become differentiable torch operations on
batches x [B][n] (float64, CUDA):

  cons(x)  -> [B][m]   backward: J(x)^T v           (exago_eval_jtv)
                       double backward: (sum_i v_i grad^2 c_i) w   (exago_eval_hvp, sigma = 0)
                                        and J(x) w                 (exago_eval_jvp)
  obj(x)   -> [B]      backward: grad f(x) scaled   (exago_eval_grad)
                       double backward: grad^2 f w  (exago_eval_hvp, lambda = 0, sigma = 1)

Every product runs in the library's kernels; torch only holds the tensors.  Third derivatives
are not provided (the second-order backward functions are marked once-differentiable).
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import exago


def _empty(B, k, like):
    return torch.empty(B, k, dtype=torch.float64, device=like.device)


def _batch(x, lam=None, mask=None, pd_scale=None, obj_weight=None, sigma=1.0):
    return exago.make_batch(x, lam, mask, pd_scale, obj_weight, sigma)


class AcopfCons(torch.autograd.Function):
    """c(x) = [g(x); h(x)] for a batch of states (mask / pd_scale are constants)."""

    @staticmethod
    def forward(ctx, x, net, mask=None, pd_scale=None):
        x = x.contiguous()
        gh = _empty(x.shape[0], net.m, x)
        exago.exago_eval_cons(net.h, _batch(x, None, mask, pd_scale), gh)
        ctx.save_for_backward(x)
        ctx.net, ctx.mask = net, mask
        return gh

    @staticmethod
    def backward(ctx, v):
        (x,) = ctx.saved_tensors
        return AcopfJtv.apply(x, v.contiguous(), ctx.net, ctx.mask), None, None, None


class AcopfJtv(torch.autograd.Function):
    """J(x)^T v; differentiable once more in both x and v."""

    @staticmethod
    def forward(ctx, x, v, net, mask=None):
        out = _empty(x.shape[0], net.n, x)
        exago.exago_eval_jtv(net.h, _batch(x, None, mask), v, out)
        ctx.save_for_backward(x, v)
        ctx.net, ctx.mask = net, mask
        return out

    @staticmethod
    @once_differentiable
    def backward(ctx, w):
        x, v = ctx.saved_tensors
        w = w.contiguous()
        net, mask = ctx.net, ctx.mask
        gx = gv = None
        if ctx.needs_input_grad[0]:
            # d/dx <w, J(x)^T v> = (sum_i v_i grad^2 c_i(x)) w: the Hessian of v^T c, sigma = 0
            gx = _empty(x.shape[0], net.n, x)
            exago.exago_eval_hvp(net.h, _batch(x, v, mask, sigma=0.0), w, gx)
        if ctx.needs_input_grad[1]:
            gv = _empty(x.shape[0], net.m, x)
            exago.exago_eval_jvp(net.h, _batch(x, None, mask), w, gv)
        return gx, gv, None, None


class AcopfObj(torch.autograd.Function):
    """f(x) per state (obj_weight = pi_s, or None for 1)."""

    @staticmethod
    def forward(ctx, x, net, obj_weight=None):
        x = x.contiguous()
        f = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        exago.exago_eval_obj(net.h, _batch(x, obj_weight=obj_weight), f)
        ctx.save_for_backward(x)
        ctx.net, ctx.w = net, obj_weight
        return f

    @staticmethod
    def backward(ctx, gf):
        (x,) = ctx.saved_tensors
        g = AcopfGrad.apply(x, ctx.net, ctx.w)
        return gf.contiguous()[:, None] * g, None, None


class AcopfGrad(torch.autograd.Function):
    """grad f(x); its backward is the objective Hessian (diagonal in Pg) times the cotangent."""

    @staticmethod
    def forward(ctx, x, net, obj_weight=None):
        g = _empty(x.shape[0], net.n, x)
        exago.exago_eval_grad(net.h, _batch(x, obj_weight=obj_weight), g)
        ctx.save_for_backward(x)
        ctx.net, ctx.w = net, obj_weight
        return g

    @staticmethod
    @once_differentiable
    def backward(ctx, w):
        (x,) = ctx.saved_tensors
        net = ctx.net
        zeros = torch.zeros(x.shape[0], net.m, dtype=torch.float64, device=x.device)
        out = _empty(x.shape[0], net.n, x)
        exago.exago_eval_hvp(net.h, _batch(x, zeros, obj_weight=ctx.w, sigma=1.0), w.contiguous(), out)
        return out, None, None


def cons(x, net, mask=None, pd_scale=None):
    """Differentiable c(x) = [g; h] of a batch (see module docstring)."""
    return AcopfCons.apply(x, net, mask, pd_scale)


def obj(x, net, obj_weight=None):
    """Differentiable f(x) of a batch."""
    return AcopfObj.apply(x, net, obj_weight)
