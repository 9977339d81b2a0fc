"""HSS matrices: interpolative decomposition, randomized compression
(Algorithm 1 with the adaptive rank scheme), mat-vec, element extraction and
the ULV-like factorization and solve.

Notation follows Section 2 of the paper: a postordered binary tree; leaves
hold D_tau; non-leaves hold B_{nu1,nu2}, B_{nu2,nu1}; every node but the root
holds U_tau, V_tau with the interpolative structure U = Pi [I; E]
(eq. UVstructure) and skeleton index sets I^r, I^c.  All arrays are float64.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------
# Interpolative decomposition (Section 2.2, ID definitions; Section 5.3 rank rule)
# ----------------------------------------------------------------------------
def cpqr_rank(Y, eps):
    """Column-pivoted Householder QR of Y (d x m), stopped at the eps-rank.

    Pivot: column of largest remaining 2-norm, norms recomputed at every step,
    lowest index wins ties.  Rank: the first i with |R_{i+1,i+1}| <= eps |R_11|
    (Section 5.3), or min(d, m); k = 0 when R_11 = 0.
    Returns (k, piv, R) with R the k x m upper-trapezoidal factor in pivoted
    column order.
    """
    Y = np.array(Y, dtype=np.float64, copy=True)
    d, m = Y.shape
    piv = np.arange(m)
    kmax = min(d, m)
    r11 = 0.0
    k = kmax
    for i in range(kmax):
        norms = np.sqrt(np.sum(Y[i:, i:] ** 2, axis=0))
        j = int(np.argmax(norms))
        nrm = norms[j]
        if i == 0:
            r11 = nrm
            if r11 == 0.0:
                k = 0
                break
        elif nrm <= eps * r11:
            k = i
            break
        if j != 0:
            Y[:, [i, i + j]] = Y[:, [i + j, i]]
            piv[[i, i + j]] = piv[[i + j, i]]
        # Householder reflector for column i, rows i..d-1 (LAPACK convention)
        x = Y[i:, i].copy()
        alpha = x[0]
        beta = -np.copysign(nrm, alpha) if alpha != 0 else -nrm
        v = x / (alpha - beta)
        v[0] = 1.0
        tau = (beta - alpha) / beta
        Y[i:, i:] -= tau * np.outer(v, v @ Y[i:, i:])
        Y[i, i] = beta
        Y[i + 1:, i] = 0.0
    R = np.triu(Y[:k, :])
    return k, piv, R


def interpolative(Y, eps):
    """[X, J] = ID(Y, eps): Y ~ Y(:, J) X with X = [I, R1^-1 R2] Pi^T.

    Returns (k, piv, E) where J = piv[:k] and E = (R1^-1 R2)^T, so that the
    basis X^T = Pi [I; E] (eq. UVstructure).
    """
    k, piv, R = cpqr_rank(Y, eps)
    m = Y.shape[1]
    if k == 0:
        return 0, piv, np.zeros((m, 0))
    X = sla.solve_triangular(R[:, :k], R[:, k:], lower=False)
    return k, piv, X.T.copy()


def interp_basis(m, k, piv, E):
    """Dense U = Pi [I; E] (m x k)."""
    U = np.zeros((m, k))
    U[piv[:k], :] = np.eye(k)
    U[piv[k:], :] = E
    return U


# ----------------------------------------------------------------------------
# HSS generators, mat-vec, extraction (Section 2.1, eq. nestedUV; Section 4.5)
# ----------------------------------------------------------------------------
class HSSMatrix:
    """Generators of an HSS matrix on tree ``tree`` (front-local ranges)."""

    def __init__(self, tree):
        self.tree = tree
        n = tree.n_nodes
        self.D = [None] * n
        self.B12 = [None] * n
        self.B21 = [None] * n
        self.U = [None] * n
        self.V = [None] * n
        self.kr = [0] * n
        self.kc = [0] * n
        self.piv_r = [None] * n
        self.piv_c = [None] * n
        self.E_r = [None] * n
        self.E_c = [None] * n
        self.Ir = [None] * n
        self.Ic = [None] * n

    def rows(self, t):
        return self.tree.hi[t] - self.tree.lo[t]

    def transpose(self):
        """Generators of A^T: D^T, U <-> V, B12 <-> B21^T."""
        T = HSSMatrix(self.tree)
        for t in range(self.tree.n_nodes):
            T.D[t] = None if self.D[t] is None else self.D[t].T.copy()
            T.B12[t] = None if self.B21[t] is None else self.B21[t].T.copy()
            T.B21[t] = None if self.B12[t] is None else self.B12[t].T.copy()
            T.U[t], T.V[t] = self.V[t], self.U[t]
            T.kr[t], T.kc[t] = self.kc[t], self.kr[t]
            T.piv_r[t], T.piv_c[t] = self.piv_c[t], self.piv_r[t]
            T.E_r[t], T.E_c[t] = self.E_c[t], self.E_r[t]
            T.Ir[t], T.Ic[t] = self.Ic[t], self.Ir[t]
        return T


def vbig_t(H, t, X, trans=False):
    """(V^big_t)^T X for X over t's rows (up-sweep); trans uses U instead."""
    tr = H.tree
    W = H.U if trans else H.V
    lo = tr.lo[t]

    def up(u):
        if tr.is_leaf(u):
            return W[u].T @ X[tr.lo[u] - lo:tr.hi[u] - lo]
        c1, c2 = tr.ch[u]
        return W[u].T @ np.vstack([up(c1), up(c2)])

    return up(t)


def ubig(H, t, G, trans=False):
    """U^big_t G (down-sweep to the leaves); trans uses V instead."""
    tr = H.tree
    W = H.V if trans else H.U
    out = np.zeros((tr.hi[t] - tr.lo[t], G.shape[1]))
    lo = tr.lo[t]

    def down(u, g):
        h = W[u] @ g
        if tr.is_leaf(u):
            out[tr.lo[u] - lo:tr.hi[u] - lo] = h
            return
        c1, c2 = tr.ch[u]
        k1 = (H.kc if trans else H.kr)[c1]
        down(c1, h[:k1])
        down(c2, h[k1:])

    down(t, G)
    return out


def matmat(H, root, X, trans=False):
    """HSS product with the sub-HSS matrix rooted at ``root``:
    up-sweep w = V^T x, B couplings between siblings, down-sweep with U,
    leaves y = D x + U g ([martinsson2011fast], cited in Section 2.1).
    ``trans`` multiplies by the transpose."""
    tr = H.tree
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    lo0 = tr.lo[root]
    nodes = tr.subtree(root)
    Wu = H.V if not trans else H.U  # up-sweep basis
    Wd = H.U if not trans else H.V  # down-sweep basis
    w = {}
    for u in nodes:
        if u == root:
            continue
        if tr.is_leaf(u):
            w[u] = Wu[u].T @ X[tr.lo[u] - lo0:tr.hi[u] - lo0]
        else:
            c1, c2 = tr.ch[u]
            w[u] = Wu[u].T @ np.vstack([w[c1], w[c2]])
    Y = np.zeros((tr.hi[root] - lo0, X.shape[1]))
    g = {}
    for u in reversed(nodes):
        if tr.is_leaf(u):
            Du = H.D[u].T if trans else H.D[u]
            y = Du @ X[tr.lo[u] - lo0:tr.hi[u] - lo0]
            if u != root:
                y = y + Wd[u] @ g[u]
            Y[tr.lo[u] - lo0:tr.hi[u] - lo0] = y
            continue
        c1, c2 = tr.ch[u]
        B12 = H.B21[u].T if trans else H.B12[u]
        B21 = H.B12[u].T if trans else H.B21[u]
        g1 = B12 @ w[c2]
        g2 = B21 @ w[c1]
        if u != root:
            h = Wd[u] @ g[u]
            k1 = (H.kc if trans else H.kr)[c1]
            g1 = g1 + h[:k1]
            g2 = g2 + h[k1:]
        g[c1], g[c2] = g1, g2
    return Y


def extract(H, root, rows, cols):
    """Elements A(rows, cols) of the sub-HSS matrix rooted at ``root``
    (indices relative to its first row), by multiplication with unit vectors
    (Section 4.5).  The tree traversal is not pruned here."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    n = H.tree.hi[root] - H.tree.lo[root]
    Ecols = np.zeros((n, len(cols)))
    Ecols[cols, np.arange(len(cols))] = 1.0
    return matmat(H, root, Ecols)[rows]


def dense(H, root=None):
    root = H.tree.root if root is None else root
    n = H.tree.hi[root] - H.tree.lo[root]
    return matmat(H, root, np.eye(n))


# ----------------------------------------------------------------------------
# Algorithm 1 (HSSCompress) with the adaptive rank scheme (Sections 2.2, 2.2.1, 4.3)
# ----------------------------------------------------------------------------
class CompressStats:
    def __init__(self):
        self.rounds = 0
        self.d_final = 0
        self.ids = 0


def compress(tree, sample, extract_fn, eps, d0, dd, p=10, stats=None):
    """Randomized HSS compression of an n x n operator given by
      sample(c0, c1) -> (R, Sr, Sc): columns c0..c1-1 of R, S^r = A R and
                        S^c = A^* R (n x (c1 - c0) each, front-local rows),
      extract_fn(rows, cols) -> A(rows, cols).
    Bottom-up over the tree.  An ID "fails" when the detected rank is above
    d - p and below the node size (reading of Section 2.2.1); on any failure,
    d grows by dd, only the new columns are sampled and pushed through the
    already-compressed nodes, and the ID is retried at the failed nodes.
    d is capped at n, where every ID is accepted.
    """
    stats = stats if stats is not None else CompressStats()
    n = tree.hi[tree.root] - tree.lo[tree.root]
    H = HSSMatrix(tree)
    d_cap = n
    d = min(d0, d_cap)
    R, Sr, Sc = sample(0, d)
    done = [False] * tree.n_nodes
    Srp = [None] * tree.n_nodes  # S^r_tau after the ID (k_r x d)
    Scp = [None] * tree.n_nodes
    Rr = [None] * tree.n_nodes  # R^r_tau = V^* R^r(I_tau) (k_c x d)
    Rc = [None] * tree.n_nodes  # R^c_tau = U^* R^c(I_tau) (k_r x d)
    d_done = [0] * tree.n_nodes  # columns already pushed through a done node
    root = tree.root
    nonroot = [t for t in range(tree.n_nodes) if t != root]

    def pre_id(t, c0, c1):
        """S^r_tau, S^c_tau before the ID, columns c0..c1-1 (Alg. 1 lines for
        the leaf and non-leaf sample updates)."""
        lo, hi = tree.lo[t], tree.hi[t]
        if tree.is_leaf(t):
            Rt = R[lo:hi, c0:c1]
            sr = Sr[lo:hi, c0:c1] - H.D[t] @ Rt
            sc = Sc[lo:hi, c0:c1] - H.D[t].T @ Rt
            return sr, sc
        c1_, c2_ = tree.ch[t]
        sr = np.vstack([Srp[c1_][:, c0:c1] - H.B12[t] @ Rr[c2_][:, c0:c1],
                        Srp[c2_][:, c0:c1] - H.B21[t] @ Rr[c1_][:, c0:c1]])
        sc = np.vstack([Scp[c1_][:, c0:c1] - H.B21[t].T @ Rc[c2_][:, c0:c1],
                        Scp[c2_][:, c0:c1] - H.B12[t].T @ Rc[c1_][:, c0:c1]])
        return sr, sc

    def r_in(t, c0, c1):
        lo, hi = tree.lo[t], tree.hi[t]
        if tree.is_leaf(t):
            Rt = R[lo:hi, c0:c1]
            return Rt, Rt
        c1_, c2_ = tree.ch[t]
        return (np.vstack([Rr[c1_][:, c0:c1], Rr[c2_][:, c0:c1]]),
                np.vstack([Rc[c1_][:, c0:c1], Rc[c2_][:, c0:c1]]))

    def post_id(t, sr, sc, c0, c1):
        """S <- S(J, :) and R^r = V^* R, R^c = U^* R for columns c0..c1-1."""
        rr_in, rc_in = r_in(t, c0, c1)
        a_sr = sr[H.piv_r[t][:H.kr[t]]]
        a_sc = sc[H.piv_c[t][:H.kc[t]]]
        a_rr = H.V[t].T @ rr_in
        a_rc = H.U[t].T @ rc_in
        if c0 == 0:
            Srp[t], Scp[t], Rr[t], Rc[t] = a_sr, a_sc, a_rr, a_rc
        else:
            Srp[t] = np.hstack([Srp[t], a_sr])
            Scp[t] = np.hstack([Scp[t], a_sc])
            Rr[t] = np.hstack([Rr[t], a_rr])
            Rc[t] = np.hstack([Rc[t], a_rc])
        d_done[t] = c1

    while True:
        stats.rounds += 1
        for t in nonroot:  # postorder
            if not tree.is_leaf(t) and not all(done[c] for c in tree.ch[t]):
                continue  # blocked by a failed descendant
            if done[t]:
                if d_done[t] < d:
                    sr, sc = pre_id(t, d_done[t], d)
                    post_id(t, sr, sc, d_done[t], d)
                continue
            # first visit or retry: extraction of D / B (kept across retries)
            if tree.is_leaf(t):
                if H.D[t] is None:
                    idx = np.arange(tree.lo[t], tree.hi[t])
                    H.D[t] = extract_fn(idx, idx)
            elif H.B12[t] is None:
                c1_, c2_ = tree.ch[t]
                H.B12[t] = extract_fn(H.Ir[c1_], H.Ic[c2_])
                H.B21[t] = extract_fn(H.Ir[c2_], H.Ic[c1_])
            sr, sc = pre_id(t, 0, d)
            m, mc = sr.shape[0], sc.shape[0]  # k_r1 + k_r2 and k_c1 + k_c2 above the leaves
            kr, pr, Er = interpolative(sr.T, eps)
            kc, pc, Ec = interpolative(sc.T, eps)
            stats.ids += 2
            ok_r = kr <= d - p or kr == m or d >= d_cap
            ok_c = kc <= d - p or kc == mc or d >= d_cap
            if not (ok_r and ok_c):
                continue
            H.kr[t], H.piv_r[t], H.E_r[t] = kr, pr, Er
            H.kc[t], H.piv_c[t], H.E_c[t] = kc, pc, Ec
            H.U[t] = interp_basis(m, kr, pr, Er)
            H.V[t] = interp_basis(mc, kc, pc, Ec)
            if tree.is_leaf(t):
                idx = np.arange(tree.lo[t], tree.hi[t])
                H.Ir[t], H.Ic[t] = idx[pr[:kr]], idx[pc[:kc]]
            else:
                c1_, c2_ = tree.ch[t]
                H.Ir[t] = np.concatenate([H.Ir[c1_], H.Ir[c2_]])[pr[:kr]]
                H.Ic[t] = np.concatenate([H.Ic[c1_], H.Ic[c2_]])[pc[:kc]]
            post_id(t, sr, sc, 0, d)
            done[t] = True
        if all(done[t] for t in nonroot):
            break
        d_new = min(d + dd, d_cap)
        Rn, Srn, Scn = sample(d, d_new)
        R = np.hstack([R, Rn])
        Sr = np.hstack([Sr, Srn])
        Sc = np.hstack([Sc, Scn])
        d = d_new
    if tree.is_leaf(root):
        if H.D[root] is None:
            idx = np.arange(tree.lo[root], tree.hi[root])
            H.D[root] = extract_fn(idx, idx)
    else:
        c1_, c2_ = tree.ch[root]
        H.B12[root] = extract_fn(H.Ir[c1_], H.Ic[c2_])
        H.B21[root] = extract_fn(H.Ir[c2_], H.Ic[c1_])
    stats.d_final = d
    return H


# ----------------------------------------------------------------------------
# ULV-like factorization and solve (Section 2.3; [xia2012superfast], [FHR])
# ----------------------------------------------------------------------------
class ULVFactor:
    """ULV-like factors of the sub-HSS matrix rooted at ``root``."""

    def __init__(self, H, root):
        self.H = H
        self.root = root
        self.nodes = H.tree.subtree(root)
        n = H.tree.n_nodes
        self.m = [0] * n
        self.L = [None] * n
        self.D21 = [None] * n
        self.Vtop = [None] * n
        self.Q = [None] * n
        self.Dhat = [None] * n
        self.Vhat = [None] * n
        self.lu = None


def omega_apply(piv, k, E, X):
    """Omega X with Omega = [[-E, I], [I, 0]] Pi^T (Section 2.3): the top
    m - k rows become X(nonskeleton) - E X(skeleton), the bottom k rows the
    skeleton rows."""
    Xp = X[piv]
    return np.vstack([Xp[k:] - E @ Xp[:k], Xp[:k]])


def ulv_factor(H, root):
    """Postorder over the subtree: Omega to zero the off-diagonal block rows,
    LQ of the top rows, reduced (D^, V^) passed to the parent; full LU at
    ``root``."""
    tr = H.tree
    F = ULVFactor(H, root)
    for t in F.nodes:
        if tr.is_leaf(t):
            Dt = H.D[t]
            Vm = H.V[t] if t != root else None
        else:
            c1, c2 = tr.ch[t]
            top = np.hstack([F.Dhat[c1], H.B12[t] @ F.Vhat[c2].T])
            bot = np.hstack([H.B21[t] @ F.Vhat[c1].T, F.Dhat[c2]])
            Dt = np.vstack([top, bot])
            Vm = None
            if t != root:
                Vm = sla.block_diag(F.Vhat[c1], F.Vhat[c2]) @ H.V[t]
        m = Dt.shape[0]
        F.m[t] = m
        if t == root:
            F.lu = sla.lu_factor(Dt) if m > 0 else None
            break
        k = H.kr[t]
        if k == m:  # nothing to eliminate: Omega = Pi^T only reorders the rows
            F.Dhat[t] = Dt[H.piv_r[t]]
            F.Vhat[t] = Vm
            continue
        Dt = omega_apply(H.piv_r[t], k, H.E_r[t], Dt)
        Qf, Rf = np.linalg.qr(Dt[:m - k].T, mode="complete")  # Dtop = [L 0] Qf^T
        F.L[t] = Rf[:m - k].T.copy()
        Dt = Dt @ Qf
        Vt = Qf.T @ Vm
        F.Q[t] = Qf
        F.D21[t] = Dt[m - k:, :m - k].copy()
        F.Vtop[t] = Vt[:m - k].copy()
        F.Dhat[t] = Dt[m - k:, m - k:].copy()
        F.Vhat[t] = Vt[m - k:].copy()
    return F


def ulv_solve(F, b):
    """x = A^-1 b with the ULV-like factors: forward elimination up the tree,
    root LU solve, backward substitution down the tree."""
    H, tr, root = F.H, F.H.tree, F.root
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    if vec:
        b = b[:, None]
    lo0 = tr.lo[root]
    nr = b.shape[1]
    bhat, w, x1 = {}, {}, {}
    z = None
    for t in F.nodes:
        if tr.is_leaf(t):
            bt = b[tr.lo[t] - lo0:tr.hi[t] - lo0]
            wc = None
        else:
            c1, c2 = tr.ch[t]
            bt = np.vstack([bhat[c1] - H.B12[t] @ w[c2], bhat[c2] - H.B21[t] @ w[c1]])
            wc = np.vstack([w[c1], w[c2]])
        if t == root:
            z = sla.lu_solve(F.lu, bt) if F.m[t] > 0 else bt
            break
        m, k = F.m[t], H.kr[t]
        wt = H.V[t].T @ wc if wc is not None else np.zeros((H.kc[t], nr))
        if k == m:
            bhat[t] = bt[H.piv_r[t]]
            w[t] = wt
            continue
        bo = omega_apply(H.piv_r[t], k, H.E_r[t], bt)
        x1[t] = sla.solve_triangular(F.L[t], bo[:m - k], lower=True)
        bhat[t] = bo[m - k:] - F.D21[t] @ x1[t]
        w[t] = wt + F.Vtop[t].T @ x1[t]
    x = np.zeros_like(b)
    xs = {root: z}
    for t in reversed(F.nodes):
        xt = xs[t]
        if t != root and F.m[t] != H.kr[t]:
            xt = F.Q[t] @ np.vstack([x1[t], xt])
        if tr.is_leaf(t):
            x[tr.lo[t] - lo0:tr.hi[t] - lo0] = xt
        else:
            c1, c2 = tr.ch[t]
            k1 = H.kr[c1]
            xs[c1], xs[c2] = xt[:k1], xt[k1:]
    return x[:, 0] if vec else x
