"""The matrix sign function by the Newton-Schulz iteration of Eq. 3,

    X_{n+1} = 1/2 X_n (3I - X_n^2),

which converges to sign(X_0) when the spectrum of X_0 lies in (-1, 1) away
from 0 (Sec. 1: the density matrix of linear-scaling DFT comes from the sign
function, two filtered multiplies per iteration). Every step runs on the device
through libbsm: 3I - X^2 is one multiply with C_in = 3I, alpha = -1, beta = 1;
the update is a second multiply with alpha = 1/2; the optional post filter
drops small blocks after each iteration, as the application does.
"""
from __future__ import annotations

import numpy as np

from .bsm import BSM_PREC_FP64, Context, Matrix


def block_identity(ctx: Context, sizes, scale: float = 1.0) -> Matrix:
    sizes = np.asarray(sizes, np.int32)
    n = len(sizes)
    vals = np.concatenate([scale * np.eye(s).reshape(-1) for s in sizes]) if n else np.zeros(0)
    idx = np.arange(n, dtype=np.int32)
    return ctx.matrix(sizes, sizes, idx, idx, vals)


def sign_iteration(ctx: Context, X0: Matrix, sizes, iters: int, eps: float = 0.0,
                   filter_eps: float | None = None, precision: int = BSM_PREC_FP64) -> Matrix:
    """Runs `iters` Newton-Schulz iterations from X0 (left untouched) and returns
    the last iterate as a new matrix on the device. `sizes` are the block sizes
    of the square matrix; eps is the on-the-fly filter of both multiplies."""
    sizes = np.asarray(sizes, np.int32)
    X = X0
    for _ in range(iters):
        T = block_identity(ctx, sizes, 3.0)
        ctx.multiply(-1.0, X, X, 1.0, T, eps, precision=precision)  # T = 3I - X^2
        Xn = ctx.empty(sizes, sizes)
        ctx.multiply(0.5, X, T, 0.0, Xn, eps, precision=precision)  # X T / 2
        if filter_eps is not None:
            Xn.filter(filter_eps)
        T.destroy()
        if X is not X0:
            X.destroy()
        X = Xn
    return X
