"""Differentiable Wilson-Dirac apply and solve for torch.autograd.

The paper evaluates D (Eq. 1) and solves D^dag D x = eta (Algorithm 1); it does not
differentiate them.  These functions add the adjoint passes so that a loss built on D psi or
on the solution x can be differentiated with respect to the spinor and the links.  All
arithmetic runs in the library's kernels; this module only allocates and calls.

Fields are complex128 CUDA tensors: spinors (V, 4, 3), links (V, 4, 3, 3), lexicographic
site order (x fastest).  Gradients follow PyTorch's convention for complex inputs,
grad = dL/dRe + i dL/dIm, so for out = D psi and an incoming gradient g:
    grad psi = D^dag g,       grad U = G(g, psi),
where G(g, psi) is the link gradient of Re <g, D psi> (lq_link_grad).  For
x = (D^dag D)^{-1} eta and incoming gradient chi, with y = (D^dag D)^{-1} chi:
    grad eta = y,             grad U = -[ G(D x, y) + G(D y, x) ].
The mass m_q is a constant (no gradient).
"""
from __future__ import annotations

import torch

from . import cg_solve, dslash_adjoint, dslash_apply, link_grad

__all__ = ["dirac_apply", "dirac_solve"]


def _volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def _spinor(buf, dims):
    return buf.view(torch.complex128).reshape(_volume(dims), 4, 3)


def _links(buf, dims):
    return buf.view(torch.complex128).reshape(_volume(dims), 4, 3, 3)


def _dense(t):
    """Materialise lazy conjugate / negative views (autograd hands those out) as plain memory."""
    return t.resolve_conj().resolve_neg().contiguous()


def _check_fields(dims, U, psi):
    V = _volume(dims)
    if U.dtype != torch.complex128 or psi.dtype != torch.complex128:
        raise TypeError("U and psi must be complex128")
    if U.shape != (V, 4, 3, 3) or psi.shape != (V, 4, 3):
        raise ValueError(f"expected U {(V, 4, 3, 3)} and psi {(V, 4, 3)}, got {tuple(U.shape)}, {tuple(psi.shape)}")


class _DiracApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, psi, dims, m_q, dagger):
        U = _dense(U)
        psi = _dense(psi)
        fn = dslash_adjoint if dagger else dslash_apply
        out = _spinor(fn(dims, m_q, U, psi), dims)
        ctx.save_for_backward(U, psi)
        ctx.dims, ctx.m_q, ctx.dagger = tuple(dims), float(m_q), bool(dagger)
        return out

    @staticmethod
    def backward(ctx, g):
        U, psi = ctx.saved_tensors
        dims, m_q, dagger = ctx.dims, ctx.m_q, ctx.dagger
        g = _dense(g)
        grad_U = grad_psi = None
        if ctx.needs_input_grad[1]:
            fn = dslash_apply if dagger else dslash_adjoint
            grad_psi = _spinor(fn(dims, m_q, U, g), dims)
        if ctx.needs_input_grad[0]:
            # Re <g, D^dag psi> = Re <psi, D g>: the same gradient with the roles swapped
            a, b = (psi, g) if dagger else (g, psi)
            grad_U = _links(link_grad(dims, a, b), dims)
        return grad_U, grad_psi, None, None, None


class _DiracSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, eta, dims, m_q, mode, tol, max_iter):
        U = _dense(U)
        eta = _dense(eta)
        x, _, st = cg_solve(dims, m_q, U, eta, mode=mode, tol=tol, max_iter=max_iter)
        if st != 0:
            raise RuntimeError(f"forward solve did not converge to {tol} in {max_iter} iterations")
        ctx.save_for_backward(U, x)
        ctx.dims, ctx.m_q, ctx.mode, ctx.tol, ctx.max_iter = tuple(dims), float(m_q), mode, tol, max_iter
        return x

    @staticmethod
    def backward(ctx, chi):
        U, x = ctx.saved_tensors
        dims, m_q = ctx.dims, ctx.m_q
        y, _, st = cg_solve(dims, m_q, U, _dense(chi), mode=ctx.mode, tol=ctx.tol, max_iter=ctx.max_iter)
        if st != 0:
            raise RuntimeError(f"adjoint solve did not converge to {ctx.tol} in {ctx.max_iter} iterations")
        grad_U = None
        if ctx.needs_input_grad[0]:
            Dx = dslash_apply(dims, m_q, U, x)
            Dy = dslash_apply(dims, m_q, U, y)
            out = link_grad(dims, Dx, y, scale=-1.0)
            link_grad(dims, Dy, x, out=out, scale=-1.0, accumulate=True)
            grad_U = _links(out, dims)
        grad_eta = y if ctx.needs_input_grad[1] else None
        return grad_U, grad_eta, None, None, None, None, None


def dirac_apply(dims, m_q, U, psi, dagger=False):
    """D psi (or D^dag psi) of Eq. (1), differentiable in U and psi."""
    _check_fields(dims, U, psi)
    return _DiracApply.apply(U, psi, tuple(dims), float(m_q), bool(dagger))


def dirac_solve(dims, m_q, U, eta, mode="mixed_f32", tol=1e-10, max_iter=100000):
    """x = (D^dag D)^{-1} eta by Algorithm 1, differentiable in U and eta.  The adjoint pass
    runs one more solve (same mode and tolerance), two applies of D and two link gradients;
    the gradient is as accurate as the two solves.  The mixed modes rebuild the inner loop's
    third link row from SU(3) unitarity; for links off SU(3) use "f64" or "f64x"."""
    _check_fields(dims, U, eta)
    return _DiracSolve.apply(U, eta, tuple(dims), float(m_q), mode, float(tol), int(max_iter))
