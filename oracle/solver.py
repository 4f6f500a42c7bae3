"""Solvers (test infrastructure; oracle).

Sec. 2.2: every inversion M s = eta (Eq. etaToS) is done with Conjugate Gradient;
a low-precision (LP) solve stops when the CG residual |r_hat| drops below a loose
bound (10^-2), a high-precision (HP) solve at a tight one.  Reading: CG on the
normal equations of the even-odd system (App. A, Eq. A.2),
    Mhat^dagger Mhat x = Mhat^dagger bhat,  x_0 = 0,
stopping when |r| / |Mhat^dagger bhat| < tol, r the CG residual of that system.
"""
from __future__ import annotations

import numpy as np

from . import operator as op


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_a, b, tol, maxiter=100000):
    """Plain CG for a hermitian positive definite operator; returns (x, iters, relres)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    bnorm = np.sqrt(rr)
    if bnorm == 0.0:
        return x, 0, 0.0
    for k in range(1, maxiter + 1):
        ap = apply_a(p)
        alpha = rr / vdot(p, ap).real
        x = x + alpha * p
        r = r - alpha * ap
        rr_new = vdot(r, r).real
        if np.sqrt(rr_new) <= tol * bnorm:
            return x, k, np.sqrt(rr_new) / bnorm
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxiter, np.sqrt(rr) / bnorm


def solve_eo(links, b, kappa, amu, f=1, bc=-1.0, tol=1e-12, maxiter=100000):
    """psi with M_f psi = b via CGNR on the even-odd system, then Eq. (A.4)."""
    dims = (links.shape[3], links.shape[2], links.shape[1], links.shape[0])
    bhat = op.prep_source(links, b, kappa, amu, f, bc, dims)
    rhs = op.mhat_dag(links, bhat, kappa, amu, f, bc, dims)

    def normal(v):
        return op.mhat_dag(links, op.mhat(links, v, kappa, amu, f, bc, dims), kappa, amu, f, bc, dims)

    x, iters, relres = cg(normal, rhs, tol, maxiter)
    psi_o = op.reconstruct_odd(links, x, b, kappa, amu, f, bc, dims)
    return x + psi_o, iters, relres


def solve_dense(links, b, kappa, amu, f=1, bc=-1.0):
    """Exact M_f^{-1} b by LU (LAPACK) of the dense matrix; small volumes only."""
    m = op.dense_matrix(links, kappa, amu, f, bc)
    return np.linalg.solve(m, b.reshape(-1)).reshape(b.shape)
