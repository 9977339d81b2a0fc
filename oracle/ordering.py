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

General sparse patterns (no geometry; the paper orders its application
matrices with METIS/SCOTCH, which are not used): ``algebraic_nested_dissection``
(level-structure separators, rule in its docstring) or a caller-given ordering
and separator tree (``fronts_from_tree``); F11 trees halve the separator's
index range.  Pinned by validity against brute-force elimination and by exact
solves (tests), and matched bit for bit by the library.
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


# ----------------------------------------------------------------------------
# General sparse patterns (no geometry)
# ----------------------------------------------------------------------------
def _halving_pieces(n, b):
    """F11 cluster tree of a separator without geometry: halve the index
    range (left part floor(n/2)) until a piece has at most b indices."""
    if n <= b:
        return ("leaf", n)
    return ("split", _halving_pieces(n // 2, b), _halving_pieces(n - n // 2, b))


def algebraic_nested_dissection(A_natural, nd_leaf=8, hss_leaf=128):
    """Nested dissection of a structurally symmetric pattern by level
    structures (a reading: the paper orders its application matrices with
    METIS/SCOTCH, which are not used here).

    - Connected components are separate elimination trees, in the order of
      their smallest vertex.
    - A set of at most max(16, nd_leaf^2) vertices is a leaf front.
    - A connected set: breadth-first search (neighbours in CSR order) from
      its first vertex; a second search from the last vertex reached gives
      the level structure.  Depth < 2: one leaf front.  Otherwise the
      separator level l is the first level >= 1 where the count of levels
      0..l passes half the set (l <= depth - 1); a level-l vertex with no
      neighbour beyond l joins the near side.  Near side, far side and
      separator keep the search order.
    - A disconnected set: its components (searched from each vertex in set
      order) sorted by decreasing size (ties in discovery order), each given
      to the group with fewer vertices so far (the first group on a tie);
      the last vertex of the second group is the separator.
    Fronts in postorder (near side, far side, separator); returns (perm,
    fronts) with perm[new] = old."""
    A = A_natural.tocsr()
    n = A.shape[0]
    rp, ci = A.indptr, A.indices
    leaf_max = max(16, nd_leaf * nd_leaf)
    perm, fronts = [], []

    def bfs(start, inset):
        order, lev = [start], {start: 0}
        h = 0
        while h < len(order):
            u = order[h]
            h += 1
            for w in ci[rp[u]:rp[u + 1]]:
                w = int(w)
                if w in inset and w not in lev:
                    lev[w] = lev[u] + 1
                    order.append(w)
        return order, lev

    def components(V):
        inset, seen, comps = set(V), set(), []
        for v in V:
            if v not in seen:
                order, _ = bfs(v, inset)
                seen.update(order)
                comps.append(order)
        return comps

    def add_front(sep, kids):
        f = Front(sep_begin=len(perm), sep_end=len(perm) + len(sep), children=list(kids))
        perm.extend(sep)
        f.sep_pieces = _halving_pieces(f.ns, hss_leaf)
        f.first = min([fronts[k].first for k in kids] + [f.sep_begin])
        fronts.append(f)
        me = len(fronts) - 1
        for k in kids:
            fronts[k].parent = me
        return me

    def rec(V):
        if len(V) <= leaf_max:
            return add_front(V, [])
        inset = set(V)
        order, lev = bfs(V[0], inset)
        if len(order) < len(V):
            comps = sorted(components(V), key=len, reverse=True)  # stable
            ga, gb, na, nb = [], [], 0, 0
            for c in comps:
                if na <= nb:
                    ga += c
                    na += len(c)
                else:
                    gb += c
                    nb += len(c)
            S = [gb.pop()]
            near, far = ga, gb
        else:
            order, lev = bfs(order[-1], inset)
            depth = lev[order[-1]]
            if depth < 2:
                return add_front(V, [])
            cnt = np.bincount([lev[v] for v in order], minlength=depth + 1)
            l, cum = 1, int(cnt[0])
            while l < depth - 1 and 2 * (cum + int(cnt[l])) <= len(V):
                cum += int(cnt[l])
                l += 1
            near, S, far = [], [], []
            for v in order:
                if lev[v] < l:
                    near.append(v)
                elif lev[v] > l:
                    far.append(v)
                elif any(int(w) in lev and lev[int(w)] > l for w in ci[rp[v]:rp[v + 1]]):
                    S.append(v)
                else:
                    near.append(v)
        kids = []
        if near:
            kids.append(rec(near))
        if far:
            kids.append(rec(far))
        return add_front(S, kids)

    for comp in components(list(range(n))):
        rec(comp)
    return np.asarray(perm, dtype=np.int64), fronts


def fronts_from_tree(n, sep_ptr, parent, hss_leaf=128):
    """Fronts of a caller-given separator tree: front f owns the new indices
    [sep_ptr[f], sep_ptr[f+1]), parent[f] > f or -1 (postorder)."""
    nf = len(parent)
    if sep_ptr[0] != 0 or sep_ptr[nf] != n:
        raise ValueError("sep_ptr must run from 0 to n")
    fronts = [Front(sep_begin=int(sep_ptr[f]), sep_end=int(sep_ptr[f + 1]), children=[]) for f in range(nf)]
    for f in range(nf):
        if fronts[f].ns < 1:
            raise ValueError("empty separator")
        p = int(parent[f])
        if p != -1 and not f < p < nf:
            raise ValueError("fronts must be in postorder")
        fronts[f].parent = p
        if p >= 0:
            fronts[p].children.append(f)
        fronts[f].sep_pieces = _halving_pieces(fronts[f].ns, hss_leaf)
    for f in range(nf):
        if len(fronts[f].children) > 2:
            raise ValueError("at most two children per front")
        fronts[f].first = min([fronts[k].first for k in fronts[f].children] + [fronts[f].sep_begin])
    return fronts


def analyze_csr(A_natural, nd_leaf=8, hss_leaf=128, perm=None, sep_ptr=None, parent=None):
    """Symbolic phase of a general pattern: the algebraic nested dissection
    (perm None) or the caller's ordering and separator tree; then I^upd, the
    HSS trees (F11 by halving) and the permuted matrix."""
    if perm is None:
        perm, fronts = algebraic_nested_dissection(A_natural, nd_leaf, hss_leaf)
    else:
        perm = np.asarray(perm, dtype=np.int64)
        if sorted(perm.tolist()) != list(range(A_natural.shape[0])):
            raise ValueError("perm is not a permutation")
        fronts = fronts_from_tree(A_natural.shape[0], sep_ptr, parent, hss_leaf)
    Anew = permute_csr(A_natural, perm)
    symbolic(fronts, Anew)
    for f in fronts:
        if f.parent >= 0:
            p = fronts[f.parent]
            if not set(f.upd.tolist()) <= set(p.indices.tolist()):
                raise ValueError("a front's I^upd is not inside its parent's index set")
        elif f.nu:
            raise ValueError("a root front has a non-empty I^upd")
    build_hss_trees(fronts, hss_leaf)
    return perm, fronts, Anew
