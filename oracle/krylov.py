"""Outer iterations around the multifrontal factorization (Section 4.6 and
the solver settings of Section 6.1).

The paper precondition GMRES(30) with modified Gram-Schmidt and a zero
initial guess when HSS compression is on, and uses iterative refinement
otherwise.  Reading taken for the stopping test: the true relative residual
||b - A x||_2 / ||b||_2 <= rtol.  Right preconditioning makes the GMRES
residual estimate that residual; it is confirmed by an explicit product
before returning.  Several right-hand sides are independent problems.
"""
from __future__ import annotations

import numpy as np


def iterative_refinement(A, apply_minv, b, rtol=1e-10, maxit=50):
    """x_0 = M^-1 b, x_{j+1} = x_j + M^-1 (b - A x_j) until converged.
    Returns (x, iterations, relres)."""
    b = np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)
    x = apply_minv(b)
    it = 1
    while True:
        r = b - A @ x
        rel = np.linalg.norm(r) / bn if bn > 0 else 0.0
        if rel <= rtol or it >= maxit:
            return x, it, rel
        x = x + apply_minv(r)
        it += 1


def gmres(A, apply_minv, b, rtol=1e-10, restart=30, maxit=300):
    """Right-preconditioned restarted GMRES with modified Gram-Schmidt,
    x_0 = 0 (Section 6.1).  Preconditioned directions z_j = M^-1 v_j are kept
    so the update is x += Z y.  Returns (x, preconditioner applications,
    relres)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bn = np.linalg.norm(b)
    x = np.zeros(n)
    if bn == 0:
        return x, 0, 0.0
    its = 0
    r = b.copy()
    beta = np.linalg.norm(r)
    while True:
        V = np.zeros((n, restart + 1))
        Z = np.zeros((n, restart))
        Hm = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        j_end = 0
        for j in range(restart):
            Z[:, j] = apply_minv(V[:, j])
            its += 1
            w = A @ Z[:, j]
            for i in range(j + 1):  # modified Gram-Schmidt
                Hm[i, j] = w @ V[:, i]
                w = w - Hm[i, j] * V[:, i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0:
                V[:, j + 1] = w / Hm[j + 1, j]
            for i in range(j):  # previous Givens rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j] = Hm[j, j] / den if den != 0 else 1.0
            sn[j] = Hm[j + 1, j] / den if den != 0 else 0.0
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j_end = j + 1
            if abs(g[j + 1]) <= rtol * bn or its >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:j_end, :j_end]), g[:j_end])
        x = x + Z[:, :j_end] @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= rtol * bn or its >= maxit:
            return x, its, beta / bn


def solve(A, apply_minv, B, use_gmres, rtol=1e-10, restart=30, maxit=300):
    """Column-by-column outer solve of A X = B; returns (X, its, relres)."""
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    X = np.zeros_like(B)
    its, rel = [], []
    for j in range(B.shape[1]):
        if use_gmres:
            x, it, rr = gmres(A, apply_minv, B[:, j], rtol, restart, maxit)
        else:
            x, it, rr = iterative_refinement(A, apply_minv, B[:, j], rtol, maxit)
        X[:, j] = x
        its.append(it)
        rel.append(rr)
    return (X[:, 0] if vec else X), its, rel
