"""General sparse matrices (hssmf_analyze_csr): the algebraic nested
dissection with dense and HSS fronts, and a caller-supplied ordering, through
factor, solve and solve_T."""
import numpy as np
import pytest

import problems

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")
spatial = pytest.importorskip("scipy.spatial")


def _geometric_operator(n, radius, seed, nonsym=False):
    """Weighted graph Laplacian of a random geometric graph in the unit cube
    plus a diagonal shift (SPD); with nonsym, off-diagonal weights differ
    between (i, j) and (j, i) (same pattern, diagonally dominant)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    pairs = spatial.cKDTree(pts).query_pairs(radius, output_type="ndarray")
    w = rng.uniform(0.5, 2.0, len(pairs))
    wt = w * rng.uniform(0.5, 1.5, len(pairs)) if nonsym else w
    rows = np.concatenate([pairs[:, 0], pairs[:, 1]])
    cols = np.concatenate([pairs[:, 1], pairs[:, 0]])
    vals = -np.concatenate([w, wt])
    L = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    d = -np.asarray(L.sum(axis=1)).ravel() + rng.uniform(0.01, 0.1, n)
    M = (L + sp.diags(d)).tocsr()
    M.sort_indices()
    return problems.CSR(n, M.indptr, M.indices, M.data), M


def _solver(**kw):
    import paper_1502_07405_gb300 as P
    return P.Solver(P.Options.defaults(**kw))


KW = dict(hss_min_front=128, hss_leaf=32, d0=32, dd=16)


def test_algebraic_order_tiny_eps_is_the_direct_solution():
    A, M = _geometric_operator(4000, 0.085, 3)
    s = _solver(hss_tol=1e-12, maxit=0, **KW)
    s.analyze_csr(A.rowptr, A.colind)
    assert s.get_stats()["n_hss_fronts"] > 10
    s.factor(A.values)
    b = problems.rhs_uniform(A.n, 2, 1)
    x = s.solve(b)
    xd = spla.spsolve(M.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("prec", [0, 1])
def test_algebraic_order_gmres_to_1e10_solve_and_solve_T(prec):
    A, M = _geometric_operator(8000, 0.07, 5, nonsym=True)
    s = _solver(hss_tol=1e-3, precision=prec, **KW)
    s.analyze_csr(A.rowptr, A.colind)
    assert s.get_stats()["n_hss_fronts"] > 20
    s.factor(A.values)
    b = problems.rhs_uniform(A.n, 3, 2)
    x = s.solve(b)
    r = np.linalg.norm(b - M @ x, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(r <= 1e-10), r
    assert s.get_stats()["iterations"] >= 2  # eps = 1e-3 is not exact
    xt = s.solve_T(b)
    rt = np.linalg.norm(b - M.T @ xt, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(rt <= 1e-10), rt


def test_disconnected_pattern_is_a_forest():
    g = problems.grid_poisson((30, 30, 1))
    A2, _ = _geometric_operator(1500, 0.11, 7)
    iso = problems.CSR(5, np.arange(6), np.arange(5), np.full(5, 3.0))
    A = problems.block_diag([g, iso, A2])
    s = _solver(hss_tol=1e-8, **KW)
    s.analyze_csr(A.rowptr, A.colind)
    s.factor(A.values)
    b = problems.rhs_uniform(A.n, 1, 4)
    x = s.solve(b)
    assert np.linalg.norm(b - A.to_scipy() @ x) <= 1e-10 * np.linalg.norm(b)


def test_caller_ordering_equals_the_grid_analysis():
    """The grid's own nested dissection handed in as a caller ordering: the
    dense factorization and its solution are the same to the last bit."""
    dims = (24, 24, 24)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 9)
    g = _solver(maxit=0, hss_min_front=1 << 30)
    g.analyze_grid(dims, A.rowptr, A.colind)
    nf = g.get_stats()["n_fronts"]
    perm, sb, se, par, nu = g.get_symbolic(nf)
    g.factor(A.values)
    xg = g.solve(b)
    c = _solver(maxit=0, hss_min_front=1 << 30)
    c.analyze_csr(A.rowptr, A.colind, perm, np.append(sb, se[-1]), par)
    c.factor(A.values)
    xc = c.solve(b)
    assert np.array_equal(xg, xc)


def test_algebraic_order_fp64_takes_the_oracles_decisions_at_inexact_eps():
    """eps = 1e-4 (inexact: one application leaves a residual ~5e-4) on a
    nonsymmetric geometric operator ordered by the algebraic nested
    dissection: the FP64 form takes the oracle's decisions (factor_csr, same
    ordering and seed) front by front and node by node, so one application
    equals the oracle's to rounding; the FP32 form stays within 10x of the
    oracle's residual."""
    from oracle import multifrontal as mf
    import paper_1502_07405_gb300 as P
    A, M = _geometric_operator(4000, 0.085, 3, nonsym=True)
    b = problems.rhs_uniform(A.n, 1, 1)
    fo = mf.factor_csr(A.to_scipy(), mf.Options(hss_tol=1e-4, **KW))
    xo = mf.apply_inverse(fo, b)
    ro = np.linalg.norm(b[:, 0] - M @ xo[:, 0]) / np.linalg.norm(b)
    assert ro > 1e-6
    stats_o = mf.hss_stats(fo)
    s = _solver(hss_tol=1e-4, maxit=0, precision=0, **KW)
    s.set_profiling(True)
    s.analyze_csr(A.rowptr, A.colind)
    s.factor(A.values)
    st = s.get_stats()
    assert st["n_hss_fronts"] == len(stats_o)
    assert st["max_rank"] == max(r for _, _, r, _, _ in stats_o)
    assert st["adaptive_rounds"] == sum(rr - 1 for _, _, _, _, rr in stats_o)
    F = P.Solver.ID_TRACE_FIELDS
    acc = {}
    for r in s.get_id_trace():
        rec = dict(zip(F, r))
        if rec["accepted"]:
            acc.setdefault(rec["front"], []).append((rec["kr"], rec["kc"]))
    for i, *_ in stats_o:
        H = fo.data[i].H
        want = sorted((H.kr[t], H.kc[t]) for t in range(H.tree.n_nodes) if t != H.tree.root)
        assert sorted(acc[i]) == want, i
    x = s.solve(b)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    s32 = _solver(hss_tol=1e-4, maxit=0, precision=1, **KW)
    s32.analyze_csr(A.rowptr, A.colind)
    s32.factor(A.values)
    x32 = s32.solve(b)
    r32 = np.linalg.norm(b[:, 0] - M @ x32[:, 0]) / np.linalg.norm(b)
    assert r32 <= 10.0 * ro, (r32, ro)
