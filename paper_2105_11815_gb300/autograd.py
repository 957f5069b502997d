"""Differentiable least-squares solve: torch.autograd.Function over the C ABI.

forward : x = argmin ||A x - b||_2 by ``ski_solve`` (Algorithm 1); R of the
          sketch is kept for the backward pass.
backward: ``ski_solve_adjoint`` solves (A^T A) lambda = g with R reused as the
          preconditioner and returns dL/db = A lambda and
          dL/dA = r lambda^T - (A lambda) x^T (r = b - A x).
Both passes run entirely in the CUDA library.
"""
import copy

import torch

from . import (dense_matrix, ski_opts_default, ski_solve, ski_solve_adjoint, ski_solve_adjoint_batched,
               ski_solve_batched)


def make_opts(d, gamma=2.0, s=1, seed=0, premix=False, tol=1e-10, tau_r=1e-12, it_max=10000, **kw):
    o = ski_opts_default(m=max(d, int(round(gamma * d))), s=s, seed=seed, premix=int(premix), tol=tol,
                         tau_r=tau_r, it_max=it_max)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class SkiLstsq(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, b, opts):
        A = A.contiguous()
        b = b.contiguous()
        d = A.shape[1]
        x = torch.empty(d, dtype=torch.float64, device=A.device)
        R = torch.empty(d, d, dtype=torch.float64, device=A.device)
        info = ski_solve(dense_matrix(A), b, opts, x, R_out=R)
        ctx.save_for_backward(A, b, x, R)
        ctx.opts = opts
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, g):
        A, b, x, R = ctx.saved_tensors
        d = A.shape[1]
        o = copy.copy(ctx.opts)
        o.tau_r = min(o.tau_r, 1e-13)
        db = torch.empty_like(b)
        dA = torch.empty_like(A) if ctx.needs_input_grad[0] else None
        ski_solve_adjoint(dense_matrix(A), b, x, R, d, g.contiguous().to(torch.float64), dA, d, db, o)
        return dA, (db if ctx.needs_input_grad[1] else None), None


def lstsq(A, b, opts=None, **kw):
    """Differentiable x = argmin ||A x - b|| for FP64 CUDA tensors A (n x d), b (n)."""
    if opts is None:
        opts = make_opts(A.shape[1], **kw)
    return SkiLstsq.apply(A, b, opts)


class SkiLstsqBatched(torch.autograd.Function):
    """Ragged batch: forward by one ``ski_solve_batched`` call, backward by one
    ``ski_solve_adjoint_batched`` call."""

    @staticmethod
    def forward(ctx, opts, *ab):
        k = len(ab) // 2
        As = [a.contiguous() for a in ab[:k]]
        bs = [b.contiguous() for b in ab[k:]]
        xs = [torch.empty(a.shape[1], dtype=torch.float64, device=a.device) for a in As]
        Rs = [torch.empty(a.shape[1], a.shape[1], dtype=torch.float64, device=a.device) for a in As]
        infos = ski_solve_batched([dense_matrix(a) for a in As], bs, opts, xs, R_outs=Rs)
        ctx.save_for_backward(*As, *bs, *xs, *Rs)
        ctx.k = k
        ctx.opts = opts
        ctx.infos = infos
        return tuple(xs)

    @staticmethod
    def backward(ctx, *gs):
        k = ctx.k
        t = ctx.saved_tensors
        As, bs, xs, Rs = t[:k], t[k:2 * k], t[2 * k:3 * k], t[3 * k:]
        o = copy.copy(ctx.opts)
        o.tau_r = min(o.tau_r, 1e-13)
        gs = [torch.zeros_like(x) if g is None else g.contiguous().to(torch.float64) for x, g in zip(xs, gs)]
        dAs = [torch.empty_like(A) for A in As]
        dbs = [torch.empty_like(b) for b in bs]
        ski_solve_adjoint_batched([dense_matrix(A) for A in As], bs, xs, Rs, gs, dAs, dbs, o)
        return (None, *dAs, *dbs)


def lstsq_batched(As, bs, opts):
    """Differentiable ragged batch; opts.m <= 0 selects m_i = gamma d_i (gamma = -m/1000)."""
    return list(SkiLstsqBatched.apply(opts, *As, *bs))
