"""torch.autograd wrapper of the block-CG solve X = A⁻¹B.

The forward pass sets the differentiable parameters of A (the diagonal shift σ
and the coupling matrices S_b) in the library and solves with h2_block_cg; the
backward pass solves the adjoint system Aᵀ Λ = ∂L/∂X with h2_block_cg
(transposed) and obtains ∂L/∂S_b = −λ̂_t x̂_sᵀ and ∂L/∂σ = −<Λ, X>_F from
h2_adjoint_grads; ∂L/∂B = Λ.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import h2 as _h2


class H2Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, sigma, S, mat, tol, max_iter, dtype):
        _h2.h2_shift_set(mat.handle, float(sigma))
        _h2.h2_coupling_set(mat.handle, S.detach().contiguous())
        X = torch.zeros_like(B)
        res = mat.block_cg(B.detach().contiguous(), X, tol=tol, max_iter=max_iter, dtype=dtype)
        if res.status != 0:
            raise _h2.H2Error(res.status, "h2_solve (forward)", f"block CG ended with {res.status_name}")
        ctx.save_for_backward(X)
        ctx.mat, ctx.tol, ctx.max_iter, ctx.dtype = mat, tol, max_iter, dtype
        return X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        mat = ctx.mat
        Lam = torch.zeros_like(gX)
        res = mat.block_cg(gX.contiguous(), Lam, tol=ctx.tol, max_iter=ctx.max_iter, dtype=ctx.dtype,
                           transposed=True)
        if res.status != 0:
            raise _h2.H2Error(res.status, "h2_solve (adjoint)", f"block CG ended with {res.status_name}")
        need_S = ctx.needs_input_grad[2]
        need_sigma = ctx.needs_input_grad[1]
        dS, dsig = _h2.h2_adjoint_grads(mat.handle, Lam, X, dS=None if need_S else False, want_dsigma=True)
        dB = Lam if ctx.needs_input_grad[0] else None
        dsigma = torch.tensor(dsig, dtype=torch.float64, device=X.device) if need_sigma else None
        return dB, dsigma, dS, None, None, None, None


def h2_solve(B, sigma, S, mat, tol=1e-10, max_iter=50000, dtype="f64"):
    """X = A(σ, S)⁻¹ B, differentiable in B, σ (0-d tensor) and S (n_adm×k×k)."""
    return H2Solve.apply(B, sigma, S, mat, tol, max_iter, dtype)
