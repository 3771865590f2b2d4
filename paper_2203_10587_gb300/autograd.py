"""torch.autograd.Function wrappers over the C ABI's evaluation and adjoint kernels.

The constraint map c(x) = [g(x); h(x)] (ExaGO, Sec. III, eqs. (8)-(9)) and the objective f(x)
(eq. (7), weighted by pi_s for scenarios, eq. (27)) become differentiable torch operations on
batches x [B][n] (float64, CUDA):

  cons(x)  -> [B][m]   backward: J(x)^T v           (exago_eval_jtv)
                       double backward: (sum_i v_i grad^2 c_i) w   (exago_eval_hvp, sigma = 0)
                                        and J(x) w                 (exago_eval_jvp)
  obj(x)   -> [B]      backward: grad f(x) scaled   (exago_eval_grad)
                       double backward: grad^2 f w  (exago_eval_hvp, lambda = 0, sigma = 1)

  cons(x, cartesian=True)  the same for the power-balance-cartesian formulation
                       (exago_eval_cart, exago_eval_cart_jtv / _hvp / _jvp)
  coupling(x) -> [B][ng]  the ramp rows Pg(x_b) - Pg(x_parent(b)) between states (eqs. (15),
                       (20), (31)); backward: C^T v into the Pg block (exago_eval_coupling_jtv),
                       whose own backward is C w (exago_eval_coupling): linear to every order

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


def _rows(net, cartesian):
    return net.m + net.nb if cartesian else net.m


class AcopfCons(torch.autograd.Function):
    """c(x) = [g(x); h(x)] for a batch of states (mask / pd_scale are constants); cartesian=True
    takes the power-balance-cartesian formulation (x = [e | f | Pg | Qg], voltage rows last)."""

    @staticmethod
    def forward(ctx, x, net, mask=None, pd_scale=None, cartesian=False):
        x = x.contiguous()
        gh = _empty(x.shape[0], _rows(net, cartesian), x)
        bt = _batch(x, None, mask, pd_scale)
        if cartesian:
            exago.exago_eval_cart(net.h, bt, gh=gh)
        else:
            exago.exago_eval_cons(net.h, bt, gh)
        ctx.save_for_backward(x)
        ctx.net, ctx.mask, ctx.cart = net, mask, cartesian
        return gh

    @staticmethod
    def backward(ctx, v):
        (x,) = ctx.saved_tensors
        return (AcopfJtv.apply(x, v.contiguous(), ctx.net, ctx.mask, ctx.cart), None, None, None,
                None)


class AcopfJtv(torch.autograd.Function):
    """J(x)^T v; differentiable once more in both x and v."""

    @staticmethod
    def forward(ctx, x, v, net, mask=None, cartesian=False):
        out = _empty(x.shape[0], net.n, x)
        (exago.exago_eval_cart_jtv if cartesian else exago.exago_eval_jtv)(
            net.h, _batch(x, None, mask), v, out)
        ctx.save_for_backward(x, v)
        ctx.net, ctx.mask, ctx.cart = net, mask, cartesian
        return out

    @staticmethod
    @once_differentiable
    def backward(ctx, w):
        x, v = ctx.saved_tensors
        w = w.contiguous()
        net, mask, cart = ctx.net, ctx.mask, ctx.cart
        gx = gv = None
        if ctx.needs_input_grad[0]:
            # d/dx <w, J(x)^T v> = (sum_i v_i grad^2 c_i(x)) w: the Hessian of v^T c, sigma = 0
            gx = _empty(x.shape[0], net.n, x)
            (exago.exago_eval_cart_hvp if cart else exago.exago_eval_hvp)(
                net.h, _batch(x, v, mask, sigma=0.0), w, gx)
        if ctx.needs_input_grad[1]:
            gv = _empty(x.shape[0], _rows(net, cart), x)
            (exago.exago_eval_cart_jvp if cart else exago.exago_eval_jvp)(
                net.h, _batch(x, None, mask), w, gv)
        return gx, gv, None, None, None


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


def cons(x, net, mask=None, pd_scale=None, cartesian=False):
    """Differentiable c(x) = [g; h] of a batch (see module docstring); cartesian=True for the
    power-balance-cartesian formulation."""
    return AcopfCons.apply(x, net, mask, pd_scale, cartesian)


def obj(x, net, obj_weight=None):
    """Differentiable f(x) of a batch."""
    return AcopfObj.apply(x, net, obj_weight)


class CouplingRows(torch.autograd.Function):
    """r = C x for an exago.Coupling; linear, so its backward is C^T and vice versa."""

    @staticmethod
    def forward(ctx, x, cpl):
        x = x.contiguous()
        r = _empty(x.shape[0], cpl.ng, x)
        exago.exago_eval_coupling(cpl.h, x, r)
        ctx.cpl = cpl
        return r

    @staticmethod
    def backward(ctx, v):
        return CouplingT.apply(v.contiguous(), ctx.cpl), None


class CouplingT(torch.autograd.Function):
    """C^T v in the stacked variable layout [B][n] (zero outside the Pg columns)."""

    @staticmethod
    def forward(ctx, v, cpl):
        v = v.contiguous()
        out = torch.zeros(v.shape[0], cpl.n, dtype=torch.float64, device=v.device)
        exago.exago_eval_coupling_jtv(cpl.h, v, out.data_ptr() + 8 * 2 * cpl.nb, cpl.n,
                                      accumulate=False)
        ctx.cpl = cpl
        return out

    @staticmethod
    def backward(ctx, w):
        return CouplingRows.apply(w.contiguous(), ctx.cpl), None


def coupling(x, cpl):
    """Differentiable coupling rows of a batch x [B][n] (cpl: exago.Coupling over B states)."""
    return CouplingRows.apply(x, cpl)
