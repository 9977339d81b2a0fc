"""Host-side checks of the CUDA library that need no GPU: it loads, exports
every entry point of include/*.h, and its symbolic phase (geometric nested
dissection, separator reordering, I^upd) agrees bit for bit with the
oracle's."""
import glob
import os
import re

import numpy as np
import pytest

import problems
from oracle import ordering

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    try:
        import paper_1502_07405_gb300 as P
    except ImportError as e:  # the build step must have run
        pytest.fail(f"library not built: {e}")
    return P


def test_exports_every_declared_symbol():
    P = _lib()
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(hssmf_[a-z_0-9A-Z]+)\s*\(", src))
    assert len(names) >= 10
    for nm in sorted(names):
        assert hasattr(P.lib, nm), nm


def test_default_opts():
    P = _lib()
    o = P.Options.defaults()
    assert o.d0 == 128 and o.dd == 64 and o.hss_leaf == 128 and o.nd_leaf == 8
    assert o.gmres_restart == 30 and o.rtol == 1e-10 and o.oversample_p == 10


@pytest.mark.parametrize("dims,leaf", [((16, 16, 1), 128), ((64, 64, 1), 128), ((33, 17, 1), 128),
                                       ((12, 10, 7), 128), ((24, 24, 24), 128), ((20, 20, 20), 32)])
def test_symbolic_bit_exact_vs_oracle(dims, leaf):
    P = _lib()
    A = problems.grid_poisson(dims)
    s = P.Solver(P.Options.defaults(hss_leaf=leaf))
    s.analyze_grid(dims, A.rowptr, A.colind)
    perm_o, fronts = ordering.nested_dissection(dims, 8, leaf)
    Anew = ordering.permute_csr(A.to_scipy(), perm_o)
    ordering.symbolic(fronts, Anew)
    perm, sb, se, par, nu = s.get_symbolic(len(fronts))
    assert np.array_equal(perm, perm_o)
    assert np.array_equal(sb, [f.sep_begin for f in fronts])
    assert np.array_equal(se, [f.sep_end for f in fronts])
    assert np.array_equal(par, [f.parent for f in fronts])
    assert np.array_equal(nu, [f.nu for f in fronts])
    for i, f in enumerate(fronts):
        assert np.array_equal(s.get_upd(i, f.nu), f.upd)
    st = s.get_stats()
    assert st["n_fronts"] == len(fronts)
    assert st["max_front"] == max(f.nf for f in fronts)


def test_analyze_rejects_bad_patterns():
    P = _lib()
    A = problems.grid_poisson((8, 8, 1))
    s = P.Solver()
    with pytest.raises(P.HssmfError):
        s.analyze_grid((8, 9, 1), A.rowptr, A.colind)  # dims do not match n
    ci = A.colind.copy()
    ci[1] = 9  # (0 -> 9) is a diagonal neighbour, (9 -> 0) is absent: not symmetric
    with pytest.raises(P.HssmfError):
        s.analyze_grid((8, 8, 1), A.rowptr, ci)
    with pytest.raises(P.HssmfError):
        s.factor(A.values)  # no successful analyze


def test_factor_before_analyze_is_an_error():
    P = _lib()
    s = P.Solver()
    with pytest.raises(P.HssmfError) as e:
        s.factor(np.zeros(5))
    assert e.value.status == P.ERR_ARG


def test_batched_grids_are_the_individual_analyses_side_by_side():
    """analyze_grids over several grids = each grid's own ordering (offset by
    the grids before it), fronts in order with parents shifted, one root per
    grid, and each grid's I^upd sizes unchanged."""
    P = _lib()
    grids = [(20, 13, 1), (9, 9, 1), (6, 7, 5), (33, 17, 1)]
    mats = [problems.grid_poisson(g) for g in grids]
    A = problems.block_diag(mats)
    s = P.Solver(P.Options.defaults(hss_leaf=32))
    s.analyze_grids(grids, A.rowptr, A.colind)
    nf_total = s.get_stats()["n_fronts"]
    perm, sb, se, par, nu = s.get_symbolic(nf_total)
    off = fo = 0
    for g, m in zip(grids, mats):
        t = P.Solver(P.Options.defaults(hss_leaf=32))
        t.analyze_grid(g, m.rowptr, m.colind)
        nf = t.get_stats()["n_fronts"]
        p1, sb1, se1, par1, nu1 = t.get_symbolic(nf)
        assert np.array_equal(perm[off:off + m.n], p1 + off)
        assert np.array_equal(sb[fo:fo + nf], sb1 + off)
        assert np.array_equal(se[fo:fo + nf], se1 + off)
        assert np.array_equal(par[fo:fo + nf], np.where(par1 >= 0, par1 + fo, -1))
        assert np.array_equal(nu[fo:fo + nf], nu1)
        off += m.n
        fo += nf
    assert fo == nf_total and off == A.n
    assert int((par < 0).sum()) == len(grids)


def test_batched_grids_reject_coupled_grids():
    P = _lib()
    A = problems.grid_poisson((8, 8, 1))
    s = P.Solver(P.Options.defaults())
    with pytest.raises(P.HssmfError):  # one 8x8 grid declared as two 8x4 grids: edges cross
        s.analyze_grids([(8, 4, 1), (8, 4, 1)], A.rowptr, A.colind)
    with pytest.raises(P.HssmfError):  # sizes do not add up
        s.analyze_grids([(8, 8, 1), (2, 2, 1)], A.rowptr, A.colind)


def _sym_pattern(n, edges):
    """CSR pattern (with diagonal) of an undirected edge list."""
    import scipy.sparse as sp
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    rows = np.concatenate([e[:, 0], e[:, 1], np.arange(n)])
    cols = np.concatenate([e[:, 1], e[:, 0], np.arange(n)])
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    M.sum_duplicates()
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32)


def _brute_force_upd(rowptr, colind, perm, sb, se):
    """I^upd of every front by the elimination game on the permuted pattern."""
    n = len(perm)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in colind[rowptr[i]:rowptr[i + 1]]:
            if i != j:
                adj[iperm[i]].add(int(iperm[j]))
    for v in range(n):  # eliminate in order: later neighbours become a clique
        later = [w for w in adj[v] if w > v]
        for a in later:
            adj[a].update(w for w in later if w != a)
    out = []
    for b, e in zip(sb, se):
        s = set()
        for v in range(b, e):
            s.update(w for w in adj[v] if w >= e)
        out.append(sorted(s))
    return out


def _random_geometric(n, radius, seed):
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    from scipy.spatial import cKDTree
    pairs = cKDTree(p).query_pairs(radius, output_type="ndarray")
    return pairs


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "geometric", "disconnected", "star", "path"])
def test_algebraic_nested_dissection_structure(case):
    """analyze_csr with no ordering: a permutation; every front's I^upd
    contains the brute-force elimination's, lies after the front's separator
    and equals it exactly where no set was split into groups of components
    (a one-vertex separator between components passes one group's I^upd
    through, which costs storage, not correctness); subtrees of sibling
    fronts joined by no edge; leaves of at most 64 vertices."""
    P = _lib()
    if case == "grid2d":
        A = problems.grid_poisson((23, 17, 1)); rp, ci = A.rowptr, A.colind
    elif case == "grid3d":
        A = problems.grid_poisson((9, 8, 7)); rp, ci = A.rowptr, A.colind
    elif case == "geometric":
        rp, ci = _sym_pattern(700, _random_geometric(700, 0.12, 1))
    elif case == "disconnected":
        g1 = problems.grid_poisson((12, 12, 1))
        g2 = problems.grid_poisson((5, 9, 1))
        iso = problems.CSR(7, np.arange(8), np.arange(7), np.ones(7))
        A = problems.block_diag([g1, iso, g2]); rp, ci = A.rowptr, A.colind
    elif case == "star":
        rp, ci = _sym_pattern(300, [(0, k) for k in range(1, 300)])
    else:
        rp, ci = _sym_pattern(500, [(k, k + 1) for k in range(499)])
    n = len(rp) - 1
    s = P.Solver(P.Options.defaults())
    s.analyze_csr(rp, ci)
    nf = s.get_stats()["n_fronts"]
    perm, sb, se, par, nu = s.get_symbolic(nf)
    assert sorted(perm.tolist()) == list(range(n))
    assert sb[0] == 0 and se[-1] == n and np.all(se > sb) and np.all(sb[1:] == se[:-1])
    upd = _brute_force_upd(rp, ci, perm, sb, se)
    for f in range(nf):  # the library's I^upd sets themselves
        lib_u = s.get_upd(f, int(nu[f])).tolist()
        assert set(upd[f]) <= set(lib_u) and all(g >= se[f] for g in lib_u)
        if case != "geometric":
            assert lib_u == upd[f]
    # leaves are small; siblings' subtrees are not adjacent
    children = [[] for _ in range(nf)]
    for f in range(nf):
        if par[f] >= 0:
            children[par[f]].append(f)
    lo = np.array(sb)
    for f in range(nf):  # subtree ranges: a front's subtree ends at its separator
        for c in children[f]:
            lo[f] = min(lo[f], lo[c])
    for f in range(nf):
        if not children[f]:
            assert se[f] - sb[f] <= 64
        if len(children[f]) == 2:
            a, b = children[f]
            va = set(perm[lo[a]:se[a]].tolist())
            vb = set(perm[lo[b]:se[b]].tolist())
            for v in va:
                assert not (set(ci[rp[v]:rp[v + 1]].tolist()) & vb)


def test_caller_ordering_reproduces_the_grid_analysis():
    P = _lib()
    dims = (20, 20, 20)
    A = problems.grid_poisson(dims)
    g = P.Solver(P.Options.defaults())
    g.analyze_grid(dims, A.rowptr, A.colind)
    nf = g.get_stats()["n_fronts"]
    perm, sb, se, par, nu = g.get_symbolic(nf)
    c = P.Solver(P.Options.defaults())
    c.analyze_csr(A.rowptr, A.colind, perm, np.append(sb, se[-1]), par)
    p2, sb2, se2, par2, nu2 = c.get_symbolic(nf)
    assert c.get_stats()["n_fronts"] == nf
    for u, v in ((perm, p2), (sb, sb2), (se, se2), (par, par2), (nu, nu2)):
        assert np.array_equal(u, v)


def test_caller_ordering_rejects_invalid_trees():
    P = _lib()
    A = problems.grid_poisson((8, 8, 1))
    n = A.n
    ident = np.arange(n)
    s = P.Solver(P.Options.defaults())
    cases = [
        (np.zeros(n), [0, n], [-1]),                        # not a permutation
        (ident, [0, 32, 32, n], [2, 2, -1]),                # empty separator
        (ident, [0, 32, n], [-1, 0]),                       # parent below child
        (ident, [0, 16, 32, 48, n], [3, 3, 3, -1]),         # three children
        (ident, [0, 32, n], [-1, -1]),                      # first half has later neighbours but is a root
    ]
    for perm, sp, pa in cases:
        with pytest.raises(P.HssmfError):
            s.analyze_csr(A.rowptr, A.colind, perm, sp, pa)
    s.analyze_csr(A.rowptr, A.colind, ident, [0, n], [-1])  # one dense front is valid


@pytest.mark.parametrize("bad", [dict(precision=2), dict(d0=0), dict(dd=0), dict(hss_tol=-1.0),
                                 dict(hss_tol=float("nan")), dict(gmres_restart=0), dict(maxit=-1),
                                 dict(hss_leaf=0), dict(nd_leaf=0), dict(oversample_p=-1)])
def test_create_rejects_bad_options(bad):
    P = _lib()
    with pytest.raises(P.HssmfError) as e:
        P.Solver(P.Options.defaults(**bad))
    assert e.value.status == P.ERR_ARG


def test_solve_and_gradient_before_factor_are_errors():
    P = _lib()
    A = problems.grid_poisson((8, 8, 1))
    s = P.Solver()
    s.analyze_grid((8, 8, 1), A.rowptr, A.colind)
    b = np.ones(A.n)
    for fn in (s.solve, s.solve_T):
        with pytest.raises(P.HssmfError) as e:
            fn(b)
        assert e.value.status == P.ERR_ARG


def test_analyze_grids_and_csr_argument_errors():
    P = _lib()
    A = problems.grid_poisson((6, 6, 1))
    s = P.Solver()
    with pytest.raises(P.HssmfError):
        s.analyze_grids([], A.rowptr, A.colind)  # no grid
    with pytest.raises(P.HssmfError):
        s.analyze_grids([(6, 0, 1)], A.rowptr, A.colind)  # empty grid
    ci = A.colind.copy()
    ci[0], ci[1] = ci[1], ci[0]  # row 0 not ascending
    with pytest.raises(P.HssmfError):
        s.analyze_csr(A.rowptr, ci)
    asym = problems.CSR(2, [0, 2, 3], [0, 1, 1], [1.0, 1.0, 1.0])  # (0, 1) without (1, 0)
    with pytest.raises(P.HssmfError):
        s.analyze_csr(asym.rowptr, asym.colind)
    one = problems.CSR(1, [0, 1], [0], [2.0])  # a 1 x 1 matrix is one leaf front
    s.analyze_csr(one.rowptr, one.colind)
    assert s.get_stats()["n_fronts"] == 1


@pytest.mark.parametrize("case", ["grid2d", "grid3d", "geometric", "disconnected", "star", "path"])
def test_algebraic_ordering_bit_exact_vs_oracle(case):
    """The library's algebraic nested dissection and symbolic phase agree
    with the oracle's bit for bit: ordering, separator ranges, parents and
    every I^upd."""
    import scipy.sparse as sp
    from oracle import ordering as ordo
    P = _lib()
    if case == "grid2d":
        A = problems.grid_poisson((23, 17, 1)); rp, ci = A.rowptr, A.colind
    elif case == "grid3d":
        A = problems.grid_poisson((9, 8, 7)); rp, ci = A.rowptr, A.colind
    elif case == "geometric":
        rp, ci = _sym_pattern(3000, _random_geometric(3000, 0.08, 2))
    elif case == "disconnected":
        g1 = problems.grid_poisson((12, 12, 1))
        g2 = problems.grid_poisson((5, 9, 1))
        iso = problems.CSR(7, np.arange(8), np.arange(7), np.ones(7))
        A = problems.block_diag([g1, iso, g2]); rp, ci = A.rowptr, A.colind
    elif case == "star":
        rp, ci = _sym_pattern(300, [(0, k) for k in range(1, 300)])
    else:
        rp, ci = _sym_pattern(500, [(k, k + 1) for k in range(499)])
    n = len(rp) - 1
    M = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    perm_o, fr_o, _ = ordo.analyze_csr(M)
    s = P.Solver(P.Options.defaults())
    s.analyze_csr(rp, ci)
    nf = s.get_stats()["n_fronts"]
    assert nf == len(fr_o)
    perm, sb, se, par, nu = s.get_symbolic(nf)
    assert np.array_equal(perm, perm_o)
    assert np.array_equal(sb, [f.sep_begin for f in fr_o])
    assert np.array_equal(se, [f.sep_end for f in fr_o])
    assert np.array_equal(par, [f.parent for f in fr_o])
    for i, f in enumerate(fr_o):
        assert np.array_equal(s.get_upd(i, f.nu), f.upd)
