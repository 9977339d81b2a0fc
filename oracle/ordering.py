"""Geometric nested dissection, separator reordering and symbolic analysis.

Paper passages followed:
  * Section 3.1 (fill-reducing nested dissection; one elimination-tree node
    per separator, Definition 1 and the amalgamation remark after it);
  * Section 6.1 (a geometric nested dissection is used for regular grids);
  * Section 4.2 (each separator is recursively bisected into pieces of about
    b = 128 vertices; each piece is an HSS leaf of F11);
  * Section 5.4 (symbolic factorization: bottom-up assembly of I^upd).

Readings where the paper is silent (all mirrored exactly by the library so
that ordering and tree agree bit for bit):
  * boxes are half-open [lo, hi) per axis; a box whose every side is
    <= nd_leaf is an elimination-tree leaf;
  * otherwise the longest side is cut (ties: lowest axis x < y < z) at
    mid = lo + len // 2; the plane coord == mid is the separator, the
    children are [lo, mid) and [mid + 1, hi);
  * numbering is postorder: left subtree, right subtree, separator;
  * the vertices of a separator (or of a leaf box) are ordered by a
    recursive bisection of its box with the same cut rule, children
    [lo, mid) and [mid, hi), until a piece has <= b vertices; pieces in
    order, x fastest inside a piece;
  * I^upd of a front: the higher-numbered vertices adjacent to its
    subtree, ascending;
  * the HSS tree of a front is root -> [F11 tree, F22 tree]; the F11 tree is
    the separator bisection tree, the F22 tree halves the sorted I^upd list
    at floor(n/2) until a node has <= b indices; a front without I^upd has
    the F11 tree as its HSS tree.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class HSSTree:
    """Binary cluster tree in postorder.  Node t covers front-local indices
    [lo[t], hi[t]); ch[t] = (left, right) or (-1, -1) for a leaf."""

    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    ch: list = field(default_factory=list)
    parent: list = field(default_factory=list)

    @property
    def n_nodes(self):
        return len(self.lo)

    @property
    def root(self):
        return self.n_nodes - 1

    def is_leaf(self, t):
        return self.ch[t][0] < 0

    def add(self, lo, hi, c1=-1, c2=-1):
        t = len(self.lo)
        self.lo.append(lo)
        self.hi.append(hi)
        self.ch.append((c1, c2))
        self.parent.append(-1)
        if c1 >= 0:
            self.parent[c1] = t
            self.parent[c2] = t
        return t

    def subtree(self, t):
        """Nodes of the subtree rooted at t, in postorder."""
        out = []

        def rec(u):
            if not self.is_leaf(u):
                rec(self.ch[u][0])
                rec(self.ch[u][1])
            out.append(u)

        rec(t)
        return out

    def depth_from_bottom(self):
        h = [0] * self.n_nodes
        for t in range(self.n_nodes):
            if not self.is_leaf(t):
                h[t] = 1 + max(h[self.ch[t][0]], h[self.ch[t][1]])
        return h


@dataclass
class Front:
    """One elimination-tree node (a separator or a leaf box)."""

    sep_begin: int
    sep_end: int
    children: list
    parent: int = -1
    sep_pieces: list = field(default_factory=list)  # nested tuples of (lo, hi) ranges
    upd: np.ndarray = None  # I^upd, ascending new indices
    first: int = 0  # first new index of the subtree
    hss: HSSTree = None
    k_node: int = -1  # F11 root inside hss
    q_node: int = -1  # F22 root inside hss (-1 if no I^upd)

    @property
    def ns(self):
        return self.sep_end - self.sep_begin

    @property
    def nu(self):
        return 0 if self.upd is None else len(self.upd)

    @property
    def nf(self):
        return self.ns + self.nu

    @property
    def indices(self):
        """I_i = [I^sep, I^upd] in new numbering."""
        return np.concatenate([np.arange(self.sep_begin, self.sep_end), self.upd])


def _cut_axis(lo, hi):
    lens = [hi[a] - lo[a] for a in range(3)]
    best = 0
    for a in (1, 2):
        if lens[a] > lens[best]:
            best = a
    return best, lens


def _box_vertices(lo, hi, nx, ny):
    """Natural indices of a box, x fastest."""
    zs = np.arange(lo[2], hi[2])
    ys = np.arange(lo[1], hi[1])
    xs = np.arange(lo[0], hi[0])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return (X + nx * (Y + ny * Z)).reshape(-1)


def _bisect_box(lo, hi, b, nx, ny, out_vertices):
    """Recursive bisection of a box into pieces of <= b vertices (Section 4.2).
    Appends the vertices in piece order to out_vertices and returns the nested
    piece structure: ('leaf', count) or ('node', left, right)."""
    vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    if vol <= b:
        out_vertices.append(_box_vertices(lo, hi, nx, ny))
        return ("leaf", vol)
    a, lens = _cut_axis(lo, hi)
    mid = lo[a] + lens[a] // 2
    hi1 = list(hi)
    hi1[a] = mid
    lo2 = list(lo)
    lo2[a] = mid
    left = _bisect_box(lo, hi1, b, nx, ny, out_vertices)
    right = _bisect_box(lo2, hi, b, nx, ny, out_vertices)
    return ("node", left, right)


def nested_dissection(dims, nd_leaf=8, hss_leaf=128):
    """Geometric nested dissection of an nx*ny*nz grid.

    Returns (perm, fronts): perm[new] = natural index; fronts in postorder
    (children before parents, the root last).
    """
    nx, ny, nz = dims
    perm_parts = []
    fronts = []
    counter = [0]

    def rec(lo, hi):
        lens = [hi[a] - lo[a] for a in range(3)]
        first = counter[0]
        if all(L <= nd_leaf for L in lens):
            verts = []
            pieces = _bisect_box(lo, hi, hss_leaf, nx, ny, verts)
            verts = np.concatenate(verts)
            f = Front(first, first + len(verts), [], sep_pieces=pieces, first=first)
            f.sep_begin = counter[0]
            counter[0] += len(verts)
            f.sep_end = counter[0]
            perm_parts.append(verts)
            fronts.append(f)
            return len(fronts) - 1
        a, _ = _cut_axis(lo, hi)
        mid = lo[a] + lens[a] // 2
        hi1 = list(hi)
        hi1[a] = mid
        lo2 = list(lo)
        lo2[a] = mid + 1
        c1 = rec(lo, hi1)
        c2 = rec(lo2, hi)
        slo = list(lo)
        shi = list(hi)
        slo[a] = mid
        shi[a] = mid + 1
        verts = []
        pieces = _bisect_box(slo, shi, hss_leaf, nx, ny, verts)
        verts = np.concatenate(verts)
        f = Front(counter[0], counter[0] + len(verts), [c1, c2], sep_pieces=pieces, first=first)
        counter[0] += len(verts)
        perm_parts.append(verts)
        fronts.append(f)
        me = len(fronts) - 1
        fronts[c1].parent = me
        fronts[c2].parent = me
        return me

    rec([0, 0, 0], [nx, ny, nz])
    perm = np.concatenate(perm_parts).astype(np.int64)
    return perm, fronts


def permute_csr(A, perm):
    """A_new = P A P^T with perm[new] = old (scipy CSR in, CSR out)."""
    A = A.tocsr()
    return A[perm][:, perm].tocsr()


def symbolic(fronts, Anew):
    """Bottom-up assembly of I^upd (Section 5.4): the neighbours of the
    separator plus the children's I^upd, restricted to indices numbered
    after the separator, in ascending order."""
    Anew = Anew.tocsr()
    for f in fronts:  # postorder
        nb = Anew.indices[Anew.indptr[f.sep_begin]:Anew.indptr[f.sep_end]]
        parts = [nb[nb >= f.sep_end]]
        for c in f.children:
            u = fronts[c].upd
            parts.append(u[u >= f.sep_end])
        f.upd = np.unique(np.concatenate(parts)).astype(np.int64)


def _pieces_to_tree(tree, pieces, offset):
    """Add the separator bisection tree to ``tree``; returns (root, size)."""
    if pieces[0] == "leaf":
        n = pieces[1]
        return tree.add(offset, offset + n), n
    l, nl = _pieces_to_tree(tree, pieces[1], offset)
    r, nr = _pieces_to_tree(tree, pieces[2], offset + nl)
    return tree.add(offset, offset + nl + nr, l, r), nl + nr


def _halving_tree(tree, lo, hi, b):
    if hi - lo <= b:
        return tree.add(lo, hi)
    mid = lo + (hi - lo) // 2
    l = _halving_tree(tree, lo, mid, b)
    r = _halving_tree(tree, mid, hi, b)
    return tree.add(lo, hi, l, r)


def build_hss_trees(fronts, hss_leaf=128):
    """Front-local HSS tree: root -> [F11 tree, F22 tree] (Sections 4.2, 4.4)."""
    for f in fronts:
        t = HSSTree()
        k, ns = _pieces_to_tree(t, f.sep_pieces, 0)
        assert ns == f.ns
        if f.nu > 0:
            q = _halving_tree(t, f.ns, f.nf, hss_leaf)
            t.add(0, f.nf, k, q)
            f.q_node = q
        else:
            f.q_node = -1
        f.k_node = k
        f.hss = t


def child_positions(fronts, c):
    """Positions of child c's I^upd inside its parent's I (the relative index
    map used by extend-add, Section 3.2)."""
    f = fronts[c]
    p = fronts[f.parent]
    I = p.indices
    pos = np.searchsorted(I[p.ns:], f.upd) + p.ns
    in_sep = (f.upd >= p.sep_begin) & (f.upd < p.sep_end)
    pos = np.where(in_sep, f.upd - p.sep_begin, pos)
    assert np.array_equal(I[pos], f.upd)
    return pos.astype(np.int64)


def etree_levels(fronts):
    """Height of each front above the leaves (leaves 0)."""
    h = [0] * len(fronts)
    for i, f in enumerate(fronts):
        if f.children:
            h[i] = 1 + max(h[c] for c in f.children)
    return h


def analyze(dims, A_natural, nd_leaf=8, hss_leaf=128):
    """Full symbolic phase: ordering, permuted matrix, I^upd, HSS trees."""
    dims = tuple(int(v) for v in dims) + (1,) * (3 - len(dims))
    perm, fronts = nested_dissection(dims, nd_leaf, hss_leaf)
    Anew = permute_csr(A_natural, perm)
    symbolic(fronts, Anew)
    build_hss_trees(fronts, hss_leaf)
    return perm, fronts, Anew
