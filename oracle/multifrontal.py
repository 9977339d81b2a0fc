"""Multifrontal LU with dense and HSS frontal matrices (Sections 3 and 4).

Dense front (Section 3.2): F_i = A_i (+) U_nu1 (+) U_nu2 (extend-add,
eq. extend-add), partial LU of F11 with row partial pivoting inside F11,
L21 = F21 U11^-1, U12 = L11^-1 P F12, update U_i = F22 - L21 U12.

HSS front (Section 4): R_i(r, c) = G(seed, I_i(r), c) (eq. Rmerge is then an
identity), samples S^r = F_i R_i and S^c = F_i^* R_i by the skinny extend-add
of eq. FtimesR, Algorithm 1 with the adaptive scheme, ULV-like factorization
of F11, low-rank Schur F21 F11^-1 F12 = Theta^* Phi (Section 4.4) with
  Z = F11^-1 U^big_k, W = (V^big_k)^* Z,
  Theta^* = U^big_q B_{q,k} W, Phi = B_{k,q} (V^big_q)^*,
where k and q are the F11 and F22 children of the front's HSS root.  The
update of an HSS front stays structured: F22 in HSS form minus Theta^* Phi,
multiplied with HSS mat-vecs and read through HSS element extraction
(Section 4.5).  A dense parent of an HSS child expands it.

Solve (Section 3.3): forward bottom-up, backward top-down.  solve_T applies
the transposed operators; HSS fronts use the ULV factorization of the
transposed HSS generators.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import hss as H_
from . import ordering
from .philox import gaussian


class Options:
    def __init__(self, hss_tol=1e-4, d0=128, dd=64, p=10, hss_min_front=1 << 30,
                 hss_leaf=128, nd_leaf=8, seed=0):
        self.hss_tol = hss_tol
        self.d0 = d0
        self.dd = dd
        self.p = p
        self.hss_min_front = hss_min_front
        self.hss_leaf = hss_leaf
        self.nd_leaf = nd_leaf
        self.seed = seed


class DenseFront:
    def __init__(self):
        self.lu = None  # LU of F11 (LAPACK layout)
        self.piv = None
        self.U12 = None
        self.L21 = None
        self.Uupd = None  # update matrix (consumed by the parent)


class HSSFront:
    def __init__(self):
        self.H = None
        self.ulv = None
        self.ulvT = None
        self.ThetaS = None
        self.Phi = None
        self.Z = None
        self.ZT = None
        self.d_final = 0
        self.rounds = 0


class Factorization:
    def __init__(self):
        self.perm = None
        self.fronts = None
        self.A = None  # permuted CSR
        self.data = []
        self.flops = 0.0
        self.t_factor = 0.0


def _front_A(Anew, f):
    """A_i: rows/cols I_i of the permuted matrix, upd x upd block removed."""
    I = f.indices
    Ai = Anew[I][:, I].tolil()
    if f.nu > 0:
        Ai[f.ns:, f.ns:] = 0.0
    return Ai.tocsr()


def _child_update_dense(fx, f):
    """Dense update matrix of a child: stored, or expanded from HSS (F22 minus
    Theta^* Phi)."""
    if isinstance(fx, DenseFront):
        return fx.Uupd
    Hc = fx.H
    return H_.dense(Hc, f.q_node) - fx.ThetaS @ fx.Phi


def extend_add(parent_n, parts):
    """Extend-add (eq. extend-add): sum of update matrices, each placed at its
    index positions of the parent's index set."""
    F = np.zeros((parent_n, parent_n))
    for pos, Uc in parts:
        F[np.ix_(pos, pos)] += Uc
    return F


def factor(A_natural, dims, opts: Options):
    """Multifrontal factorization of a matrix on a grid (geometric ND)."""
    t0 = time.perf_counter()
    perm, fronts, Anew = ordering.analyze(dims, A_natural, opts.nd_leaf, opts.hss_leaf)
    return _factor_ordered(perm, fronts, Anew, opts, t0)


def factor_subtree(A_natural, dims, opts: Options, depth):
    """Factor only the fronts of one subtree of a grid's elimination tree:
    the subtree of the front reached from the root by taking the first child
    ``depth`` times.  Every front of it is factored exactly as in the whole
    factorization (same ordering, update sets and random sketch); the other
    fronts are left out (data None).  A bounded piece of the whole workload,
    for timing the oracle.  Returns the partial factorization and the
    subtree's front indices."""
    t0 = time.perf_counter()
    perm, fronts, Anew = ordering.analyze(dims, A_natural, opts.nd_leaf, opts.hss_leaf)
    r = len(fronts) - 1
    for _ in range(depth):
        if not fronts[r].children:
            break
        r = fronts[r].children[0]
    sub, stack = {r}, [r]
    while stack:
        for c in fronts[stack.pop()].children:
            sub.add(c)
            stack.append(c)
    return _factor_ordered(perm, fronts, Anew, opts, t0, only=sub), sorted(sub)


def factor_csr(A_natural, opts: Options, perm=None, sep_ptr=None, parent=None):
    """Multifrontal factorization of a general pattern: algebraic nested
    dissection, or the caller's ordering and separator tree."""
    t0 = time.perf_counter()
    perm, fronts, Anew = ordering.analyze_csr(A_natural, opts.nd_leaf, opts.hss_leaf, perm, sep_ptr, parent)
    return _factor_ordered(perm, fronts, Anew, opts, t0)


def _factor_ordered(perm, fronts, Anew, opts, t0, only=None):
    fz = Factorization()
    fz.perm, fz.fronts, fz.A = perm, fronts, Anew
    fz.data = [None] * len(fronts)
    pos = {}
    for i, f in enumerate(fronts):
        if only is not None and i not in only:
            continue  # (a partial factorization needs only its own fronts' maps)
        for c in f.children:
            pos[c] = ordering.child_positions(fronts, c)
    for i, f in enumerate(fronts):
        if only is not None and i not in only:
            continue
        if f.nf >= opts.hss_min_front:
            fz.data[i] = _factor_hss_front(fz, i, pos, opts)
        else:
            fz.data[i] = _factor_dense_front(fz, i, pos)
    fz.t_factor = time.perf_counter() - t0
    return fz


def _factor_dense_front(fz, i, pos):
    f = fz.fronts[i]
    ns, nu = f.ns, f.nu
    Ai = _front_A(fz.A, f).toarray()
    parts = [(pos[c], _child_update_dense(fz.data[c], fz.fronts[c])) for c in f.children]
    F = Ai + extend_add(f.nf, parts)
    out = DenseFront()
    lu, piv = sla.lu_factor(F[:ns, :ns], check_finite=True)
    F12 = F[:ns, ns:].copy()
    for j in range(ns):  # row interchanges of getrf applied to F12
        if piv[j] != j:
            F12[[j, piv[j]]] = F12[[piv[j], j]]
    U12 = sla.solve_triangular(lu, F12, lower=True, unit_diagonal=True)
    L21 = sla.solve_triangular(lu, F[ns:, :ns].T, trans="T", lower=False).T
    out.lu, out.piv, out.U12, out.L21 = lu, piv, U12, L21
    out.Uupd = F[ns:, ns:] - L21 @ U12
    fz.flops += 2.0 / 3.0 * ns ** 3 + 2.0 * ns ** 2 * nu + 2.0 * ns * nu ** 2
    return out


def _factor_hss_front(fz, i, pos, opts):
    f = fz.fronts[i]
    I = f.indices
    Ai = _front_A(fz.A, f)
    AiT = Ai.T.tocsr()
    kids = []
    for c in f.children:
        inv = np.full(f.nf, -1, dtype=np.int64)
        inv[pos[c]] = np.arange(len(pos[c]))
        kids.append((pos[c], inv, fz.data[c], fz.fronts[c]))

    def child_mul(fx, fc, X, trans):
        if isinstance(fx, DenseFront):
            return (fx.Uupd.T if trans else fx.Uupd) @ X
        Y = H_.matmat(fx.H, fc.q_node, X, trans=trans)
        if trans:
            return Y - fx.Phi.T @ (fx.ThetaS.T @ X)
        return Y - fx.ThetaS @ (fx.Phi @ X)

    def sample(c0, c1):
        R = gaussian(opts.seed, I, np.arange(c0, c1))
        Sr = Ai @ R
        Sc = AiT @ R
        for p_, inv, fx, fc in kids:
            X = R[p_]
            Sr[p_] += child_mul(fx, fc, X, False)
            Sc[p_] += child_mul(fx, fc, X, True)
        return R, Sr, Sc

    def extract_fn(rows, cols):
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        out = Ai[rows][:, cols].toarray()
        for p_, inv, fx, fc in kids:
            ri, ci = inv[rows], inv[cols]
            rs, cs = np.nonzero(ri >= 0)[0], np.nonzero(ci >= 0)[0]
            if len(rs) == 0 or len(cs) == 0:
                continue
            a, b = ri[rs], ci[cs]
            if isinstance(fx, DenseFront):
                blk = fx.Uupd[np.ix_(a, b)]
            else:
                blk = H_.extract(fx.H, fc.q_node, a, b) - fx.ThetaS[a] @ fx.Phi[:, b]
            out[np.ix_(rs, cs)] += blk
        return out

    st = H_.CompressStats()
    Hm = H_.compress(f.hss, sample, extract_fn, opts.hss_tol, opts.d0, opts.dd, opts.p, st)
    out = HSSFront()
    out.H = Hm
    out.d_final, out.rounds = st.d_final, st.rounds
    k, q = f.k_node, f.q_node
    out.ulv = H_.ulv_factor(Hm, k)
    if q >= 0:
        root = f.hss.root
        Ubk = H_.ubig(Hm, k, np.eye(Hm.kr[k]))
        out.Z = H_.ulv_solve(out.ulv, Ubk)
        W = H_.vbig_t(Hm, k, out.Z)
        out.ThetaS = H_.ubig(Hm, q, Hm.B21[root] @ W)
        out.Phi = Hm.B12[root] @ H_.vbig_t(Hm, q, np.eye(f.nu))
    return out


def _ensure_transposed(fx, f):
    if fx.ulvT is None:
        HT = fx.H.transpose()
        fx.ulvT = H_.ulv_factor(HT, f.k_node)
        if f.q_node >= 0:
            fx.ZT = H_.ulv_solve(fx.ulvT, H_.ubig(fx.H, f.k_node, np.eye(fx.H.kc[f.k_node]), trans=True))


def apply_inverse(fz, b, transpose=False):
    """x = M^-1 b with the (approximate) multifrontal factorization M of the
    natural-order matrix; b is (n,) or (n, nrhs) in natural order."""
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    if vec:
        b = b[:, None]
    y = b[fz.perm].copy()
    fronts = fz.fronts
    for i, f in enumerate(fronts):  # forward, bottom-up
        fx = fz.data[i]
        if fx is None:  # a front left out of a partial factorization (factor_subtree)
            continue
        s = slice(f.sep_begin, f.sep_end)
        if isinstance(fx, DenseFront):
            ys = y[s]
            if not transpose:
                for j in range(f.ns):
                    if fx.piv[j] != j:
                        ys[[j, fx.piv[j]]] = ys[[fx.piv[j], j]]
                ys = sla.solve_triangular(fx.lu, ys, lower=True, unit_diagonal=True)
                if f.nu:
                    y[f.upd] -= fx.L21 @ ys
            else:
                ys = sla.solve_triangular(fx.lu, ys, lower=False, trans="T")
                if f.nu:
                    y[f.upd] -= fx.U12.T @ ys
            y[s] = ys
        else:
            Hm, k, q = fx.H, f.k_node, f.q_node
            if not transpose:
                ys = H_.ulv_solve(fx.ulv, y[s])
                if q >= 0:
                    root = f.hss.root
                    y[f.upd] -= H_.ubig(Hm, q, Hm.B21[root] @ H_.vbig_t(Hm, k, ys))
            else:
                _ensure_transposed(fx, f)
                ys = H_.ulv_solve(fx.ulvT, y[s])
                if q >= 0:
                    root = f.hss.root
                    y[f.upd] -= H_.ubig(Hm, q, Hm.B12[root].T @ H_.vbig_t(Hm, k, ys, trans=True), trans=True)
            y[s] = ys
    x = y
    for i in reversed(range(len(fronts))):  # backward, top-down
        f, fx = fronts[i], fz.data[i]
        if fx is None:
            continue
        s = slice(f.sep_begin, f.sep_end)
        if isinstance(fx, DenseFront):
            ys = x[s]
            if not transpose:
                if f.nu:
                    ys = ys - fx.U12 @ x[f.upd]
                x[s] = sla.solve_triangular(fx.lu, ys, lower=False)
            else:
                if f.nu:
                    ys = ys - fx.L21.T @ x[f.upd]
                z = sla.solve_triangular(fx.lu, ys, lower=True, unit_diagonal=True, trans="T")
                for j in reversed(range(f.ns)):
                    if fx.piv[j] != j:
                        z[[j, fx.piv[j]]] = z[[fx.piv[j], j]]
                x[s] = z
        else:
            Hm, k, q = fx.H, f.k_node, f.q_node
            if q < 0:
                continue
            root = f.hss.root
            if not transpose:
                x[s] = x[s] - fx.Z @ (Hm.B12[root] @ H_.vbig_t(Hm, q, x[f.upd]))
            else:
                x[s] = x[s] - fx.ZT @ (Hm.B21[root].T @ H_.vbig_t(Hm, q, x[f.upd], trans=True))
    out = np.empty_like(x)
    out[fz.perm] = x
    return out[:, 0] if vec else out


def hss_stats(fz):
    """Per-HSS-front maximum rank, final d and adaptive rounds."""
    out = []
    for i, f in enumerate(fz.fronts):
        fx = fz.data[i]
        if isinstance(fx, HSSFront):
            r = max(max(fx.H.kr), max(fx.H.kc))
            out.append((i, f.nf, r, fx.d_final, fx.rounds))
    return out
