"""Pins of the CPU oracle against facts fixed outside it: published
known-answer vectors, the paper's worked examples, textbook routines
(LAPACK through numpy/scipy), brute force on tiny inputs, closed forms and
invariants.  CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import problems
from oracle import hss, krylov, multifrontal as mf, ordering
from oracle.philox import gaussian, philox4x32_10

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    for r in _load("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        out = philox4x32_10(np.array(v[:4]), np.array(v[4:6]))
        assert [int(o) for o in out] == v[6:]


def test_gaussian_moments_and_row_consistency():
    g = gaussian(0, np.arange(2000), np.arange(500))
    assert abs(g.mean()) < 5e-3
    assert abs(g.var() - 1.0) < 1e-2
    assert abs(np.mean(g ** 4) - 3.0) < 0.05
    # Fig. extend-add: I_1 = {1,4,5}, I_2 = {2,3,4,5,7}, I_3 = {4,5,6,7};
    # entries of shared global rows agree in every front's R.
    R1 = gaussian(7, [1, 4, 5], range(1))
    R2 = gaussian(7, [2, 3, 4, 5, 7], range(2))
    R3 = gaussian(7, [4, 5, 6, 7], range(3))
    assert R1[1, 0] == R2[2, 0] == R3[0, 0]  # r_{4,1}
    assert R1[2, 0] == R2[3, 0] == R3[1, 0]  # r_{5,1}
    assert np.array_equal(R2[2:4, 1], R3[0:2, 1])  # r_{4,2}, r_{5,2}
    assert np.array_equal(R2[4, :2], R3[3, :2])  # r_{7,1}, r_{7,2}
    assert R1[0, 0] != R1[1, 0]


# ---------------------------------------------------------------- extend-add
def test_extend_add_worked_example():
    a1, b1, c1, d1, a2, b2, c2, d2 = 2, 3, 5, 7, 11, 13, 17, 19
    U1 = np.array([[a1, b1], [c1, d1]], float)
    U2 = np.array([[a2, b2], [c2, d2]], float)
    # parent index set {1,2,3}: positions of {1,2} and {1,3}
    F = mf.extend_add(3, [(np.array([0, 1]), U1), (np.array([0, 2]), U2)])
    expect = np.array(_load("extend_add_example.txt"), dtype=float)
    assert np.array_equal(F, expect)


# ------------------------------------------------------------------ ordering
def test_nd_16x16_hand_checked():
    perm, fronts = ordering.nested_dissection((16, 16, 1))
    # x cut at 8 -> 8x16 | 7x16; then y cuts at 8: leaves 8x8, 8x7, 7x8, 7x7
    assert [(f.ns, f.children) for f in fronts] == [
        (64, []), (56, []), (8, [0, 1]), (56, []), (49, []), (7, [3, 4]), (16, [2, 5])]
    assert sorted(perm.tolist()) == list(range(256))
    # the root separator is the column x = 8, ordered by y
    assert perm[-16:].tolist() == [8 + 16 * y for y in range(16)]
    # the first leaf box is x, y in [0, 8), x fastest
    assert perm[:8].tolist() == list(range(8))


@pytest.mark.parametrize("dims", [(12, 12, 1), (20, 9, 1), (7, 6, 5), (10, 10, 10)])
def test_nd_separates_and_postorders(dims):
    A = problems.grid_poisson(dims).to_scipy()
    perm, fronts, Anew = ordering.analyze(dims, A)
    Anew = Anew.tocsr()
    for i, f in enumerate(fronts):
        for c in f.children:
            assert fronts[c].sep_end <= f.sep_begin  # postorder
        if len(f.children) == 2:
            c1, c2 = (fronts[c] for c in f.children)
            s1 = np.arange(c1.first, c1.sep_end)
            s2 = np.arange(c2.first, c2.sep_end)
            assert Anew[s1][:, s2].nnz == 0  # the separator splits the subtrees


@pytest.mark.parametrize("dims", [(9, 9, 1), (12, 10, 1), (5, 5, 5)])
def test_symbolic_matches_brute_force_elimination(dims):
    A = problems.grid_poisson(dims).to_scipy()
    perm, fronts, Anew = ordering.analyze(dims, A)
    n = Anew.shape[0]
    S = (Anew.toarray() != 0)
    for j in range(n):  # boolean Gaussian elimination: fill pattern of L
        rows = np.nonzero(S[j + 1:, j])[0] + j + 1
        S[np.ix_(rows, rows)] = True
    for f in fronts:
        cols = np.arange(f.sep_begin, f.sep_end)
        below = np.nonzero(S[f.sep_end:, cols].any(axis=1))[0] + f.sep_end
        assert np.array_equal(below, f.upd)


# ------------------------------------------------------------------ dense MF
@pytest.mark.parametrize("dims", [(4, 4, 1), (8, 8, 1), (16, 16, 1), (4, 4, 4), (9, 7, 3)])
def test_dense_mf_matches_lapack(dims):
    A = problems.grid_poisson(dims).to_scipy()
    n = A.shape[0]
    b = problems.rhs_uniform(n, 2, 1)
    fz = mf.factor(A, dims, mf.Options())
    x = mf.apply_inverse(fz, b)
    xe = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xe) <= 1e-12 * np.linalg.norm(xe)
    xt = mf.apply_inverse(fz, b, transpose=True)
    assert np.linalg.norm(xt - xe) <= 1e-12 * np.linalg.norm(xe)  # symmetric A


def _random_on_pattern(dims, seed):
    A = problems.grid_poisson(dims).to_scipy().tocsr()
    rng = np.random.default_rng(seed)
    vals = rng.uniform(-1, 1, A.nnz)
    B = sp.csr_matrix((vals, A.indices, A.indptr), shape=A.shape)
    B.setdiag(rng.uniform(0.2, 1.0, A.shape[0]) * rng.choice([-1, 1], A.shape[0]))
    return B.tocsr()


@pytest.mark.parametrize("dims", [(8, 8, 1), (5, 4, 3)])
def test_dense_mf_nonsymmetric_pivoting(dims):
    A = _random_on_pattern(dims, 3)
    n = A.shape[0]
    b = problems.rhs_uniform(n, 1, 2)[:, 0]
    fz = mf.factor(A, dims, mf.Options())
    assert any((fx.piv != np.arange(len(fx.piv))).any() for fx in fz.data)  # pivoting happened
    x = mf.apply_inverse(fz, b)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    xt = mf.apply_inverse(fz, b, transpose=True)
    assert np.linalg.norm(A.T @ xt - b) <= 1e-10 * np.linalg.norm(b)


def test_ones_solution():
    dims = (16, 16, 1)
    A = problems.grid_poisson(dims).to_scipy()
    b = A @ np.ones(A.shape[0])
    fz = mf.factor(A, dims, mf.Options())
    x = mf.apply_inverse(fz, b)
    assert np.max(np.abs(x - 1.0)) < 1e-12


def test_manufactured_solution_second_order():
    errs = []
    for k in (15, 31, 63):
        h = 1.0 / (k + 1)
        A = problems.grid_poisson((k, k, 1), scale=(k + 1) ** 2).to_scipy()
        xs = np.arange(1, k + 1) * h
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        u = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
        f = 2 * np.pi ** 2 * u
        fz = mf.factor(A, (k, k, 1), mf.Options())
        errs.append(np.max(np.abs(mf.apply_inverse(fz, f) - u)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2


# ------------------------------------------------------------------------ ID
def test_id_exact_for_rank_k():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((40, 9)) @ rng.standard_normal((9, 60))
    k, piv, E = hss.interpolative(Y, 1e-12)
    assert k == 9
    X = np.zeros((k, 60))
    X[:, piv[:k]] = np.eye(k)
    X[:, piv[k:]] = E.T
    assert np.linalg.norm(Y[:, piv[:k]] @ X - Y) <= 1e-12 * np.linalg.norm(Y)


def test_id_detects_prescribed_rank():
    rng = np.random.default_rng(1)
    Q1, _ = np.linalg.qr(rng.standard_normal((80, 30)))
    Q2, _ = np.linalg.qr(rng.standard_normal((50, 30)))
    s = 10.0 ** -np.arange(30, dtype=float)
    Y = (Q1 * s) @ Q2.T
    for eps, want in [(3e-3, 3), (3e-7, 7), (3e-11, 11)]:
        k, _, _ = hss.interpolative(Y, eps)
        assert k == want


def test_cpqr_pivots_match_lapack_geqp3():
    rng = np.random.default_rng(2)
    for shape in [(30, 20), (20, 30), (64, 64)]:
        Y = rng.standard_normal(shape)
        k, piv, R = hss.cpqr_rank(Y, 0.0)
        _, Rl, pl = sla.qr(Y, pivoting=True)
        assert k == min(shape)
        assert np.array_equal(piv[:k], pl[:k])
        assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-10)


def test_id_zero_matrix_rank_zero():
    k, piv, E = hss.interpolative(np.zeros((10, 7)), 1e-6)
    assert k == 0 and E.shape == (7, 0)


# ----------------------------------------------------------------------- HSS
def _tree(n, leaf):
    t = ordering.HSSTree()
    ordering._halving_tree(t, 0, n, leaf)
    return t


def _random_hss(tree, r, rng):
    """Random generators with off-diagonal rank r (nested bases)."""
    H = hss.HSSMatrix(tree)
    for t in range(tree.n_nodes):
        m = H.rows(t) if tree.is_leaf(t) else 2 * r
        if tree.is_leaf(t):
            H.D[t] = rng.standard_normal((m, m)) + m * np.eye(m)
        else:
            H.B12[t] = rng.standard_normal((r, r))
            H.B21[t] = rng.standard_normal((r, r))
        if t != tree.root:
            H.U[t] = rng.standard_normal((m, r))
            H.V[t] = rng.standard_normal((m, r))
            H.kr[t] = H.kc[t] = r
    return H


def test_hss_matmat_matches_paper_example():
    """eq. HSSexamplematrix: the 7-node postordered tree written out block by
    block, against the generic nested-basis mat-vec."""
    rng = np.random.default_rng(3)
    t = ordering.HSSTree()
    n1 = t.add(0, 5)
    n2 = t.add(5, 9)
    n3 = t.add(0, 9, n1, n2)
    n4 = t.add(9, 15)
    n5 = t.add(15, 20)
    n6 = t.add(9, 20, n4, n5)
    t.add(0, 20, n3, n6)
    H = hss.HSSMatrix(t)
    r = {0: 2, 1: 3, 2: 2, 3: 3, 4: 2, 5: 3}
    H.D[0], H.D[1] = rng.standard_normal((5, 5)), rng.standard_normal((4, 4))
    H.D[3], H.D[4] = rng.standard_normal((6, 6)), rng.standard_normal((5, 5))
    for leaf, m in [(0, 5), (1, 4), (3, 6), (4, 5)]:
        H.U[leaf] = rng.standard_normal((m, r[leaf]))
        H.V[leaf] = rng.standard_normal((m, r[leaf]))
        H.kr[leaf] = H.kc[leaf] = r[leaf]
    for node, (a, b) in [(2, (0, 1)), (5, (3, 4))]:
        H.U[node] = rng.standard_normal((r[a] + r[b], r[node]))
        H.V[node] = rng.standard_normal((r[a] + r[b], r[node]))
        H.kr[node] = H.kc[node] = r[node]
        H.B12[node] = rng.standard_normal((r[a], r[b]))
        H.B21[node] = rng.standard_normal((r[b], r[a]))
    H.B12[6] = rng.standard_normal((r[2], r[5]))
    H.B21[6] = rng.standard_normal((r[5], r[2]))
    U, V, D, B12, B21 = H.U, H.V, H.D, H.B12, H.B21
    bd = sla.block_diag
    A = np.zeros((20, 20))
    A[0:5, 0:5] = D[0]
    A[0:5, 5:9] = U[0] @ B12[2] @ V[1].T
    A[5:9, 0:5] = U[1] @ B21[2] @ V[0].T
    A[5:9, 5:9] = D[1]
    A[0:9, 9:20] = bd(U[0], U[1]) @ U[2] @ B12[6] @ V[5].T @ bd(V[3].T, V[4].T)
    A[9:20, 0:9] = bd(U[3], U[4]) @ U[5] @ B21[6] @ V[2].T @ bd(V[0].T, V[1].T)
    A[9:15, 9:15] = D[3]
    A[9:15, 15:20] = U[3] @ B12[5] @ V[4].T
    A[15:20, 9:15] = U[4] @ B21[5] @ V[3].T
    A[15:20, 15:20] = D[4]
    X = rng.standard_normal((20, 3))
    assert np.allclose(hss.matmat(H, 6, X), A @ X, rtol=1e-13, atol=1e-12)
    assert np.allclose(hss.matmat(H, 6, X, trans=True), A.T @ X, rtol=1e-13, atol=1e-12)
    rows, cols = np.array([0, 7, 19, 3]), np.array([18, 2, 9, 5, 6])
    assert np.allclose(hss.extract(H, 6, rows, cols), A[np.ix_(rows, cols)], atol=1e-12)
    # sub-HSS rooted at node 5 is A[9:20, 9:20]
    assert np.allclose(hss.dense(H, 5), A[9:20, 9:20], atol=1e-12)


def _dense_sampler(A, seed=5):
    n = A.shape[0]

    def sample(c0, c1):
        R = gaussian(seed, np.arange(n), np.arange(c0, c1))
        return R, A @ R, A.T @ R

    return sample


def test_compress_known_rank_and_submatrix_B():
    rng = np.random.default_rng(4)
    tree = _tree(512, 64)
    A = hss.dense(_random_hss(tree, 7, rng))
    H = hss.compress(tree, _dense_sampler(A), lambda r, c: A[np.ix_(r, c)], 1e-10, 32, 16)
    for t in range(tree.n_nodes - 1):
        assert H.kr[t] == 7 and H.kc[t] == 7
    assert np.linalg.norm(hss.dense(H) - A) <= 1e-11 * np.linalg.norm(A)
    for t in range(tree.n_nodes):
        if not tree.is_leaf(t):
            c1, c2 = tree.ch[t]
            assert np.array_equal(H.B12[t], A[np.ix_(H.Ir[c1], H.Ic[c2])])  # exact submatrix
            assert np.array_equal(H.B21[t], A[np.ix_(H.Ir[c2], H.Ic[c1])])


def test_compress_exact_as_eps_to_zero_with_adaptive_d():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((200, 200))
    tree = _tree(200, 50)
    st = hss.CompressStats()
    H = hss.compress(tree, _dense_sampler(A), lambda r, c: A[np.ix_(r, c)], 1e-14, 16, 16, stats=st)
    assert st.rounds > 1  # the adaptive scheme had to grow d
    assert np.linalg.norm(hss.dense(H) - A) <= 1e-12 * np.linalg.norm(A)


def test_compress_error_tracks_eps():
    x = np.linspace(0, 1, 400)
    A = 1.0 / (np.abs(x[:, None] - x[None, :]) + 0.05)
    tree = _tree(400, 50)
    errs = []
    for eps in (1e-3, 1e-6, 1e-9):
        H = hss.compress(tree, _dense_sampler(A), lambda r, c: A[np.ix_(r, c)], eps, 40, 20)
        errs.append(np.linalg.norm(hss.dense(H) - A) / np.linalg.norm(A))
        assert errs[-1] <= 100 * eps
    assert errs[0] > errs[1] > errs[2]


def test_omega_zeroes_basis_rows():
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((12, 9)) @ rng.standard_normal((9, 20))
    k, piv, E = hss.interpolative(Y, 1e-12)
    U = hss.interp_basis(20, k, piv, E)
    OU = hss.omega_apply(piv, k, E, U)
    assert np.allclose(OU[:20 - k], 0, atol=1e-13)
    assert np.array_equal(OU[20 - k:], np.eye(k))


def test_ulv_solve_matches_dense_solve():
    rng = np.random.default_rng(8)
    x = np.linspace(0, 1, 300)
    A = 1.0 / (np.abs(x[:, None] - x[None, :]) + 0.05) + 5 * np.eye(300)
    A += 0.01 * rng.standard_normal((300, 300)) * (np.abs(x[:, None] - x[None, :]) < 0.1)
    tree = _tree(300, 40)
    H = hss.compress(tree, _dense_sampler(A), lambda r, c: A[np.ix_(r, c)], 1e-8, 40, 20)
    Ad = hss.dense(H)
    b = rng.standard_normal((300, 2))
    F = hss.ulv_factor(H, tree.root)
    xs = hss.ulv_solve(F, b)
    assert np.linalg.norm(xs - np.linalg.solve(Ad, b)) <= 1e-12 * np.linalg.norm(xs)
    FT = hss.ulv_factor(H.transpose(), tree.root)
    xt = hss.ulv_solve(FT, b)
    assert np.linalg.norm(xt - np.linalg.solve(Ad.T, b)) <= 1e-12 * np.linalg.norm(xt)


# ------------------------------------------------------------------ MF + HSS
def test_mf_hss_exact_at_tiny_eps_matches_dense_mf():
    dims = (32, 32, 1)
    A = problems.grid_poisson(dims).to_scipy()
    b = problems.rhs_uniform(A.shape[0], 1, 1)[:, 0]
    fd = mf.factor(A, dims, mf.Options())
    fh = mf.factor(A, dims, mf.Options(hss_tol=1e-14, d0=64, dd=32, hss_min_front=64))
    assert len(mf.hss_stats(fh)) > 10
    xd = mf.apply_inverse(fd, b)
    xh = mf.apply_inverse(fh, b)
    assert np.linalg.norm(xh - xd) <= 1e-10 * np.linalg.norm(xd)
    xht = mf.apply_inverse(fh, b, transpose=True)
    assert np.linalg.norm(xht - xd) <= 1e-10 * np.linalg.norm(xd)


def test_mf_hss_preconditioned_gmres_converges_3d():
    dims = (12, 12, 12)
    A = problems.grid_poisson(dims).to_scipy()
    b = problems.rhs_uniform(A.shape[0], 1, 1)[:, 0]
    fh = mf.factor(A, dims, mf.Options(hss_tol=1e-2, d0=64, dd=32, hss_min_front=200, hss_leaf=32))
    assert len(mf.hss_stats(fh)) > 0
    x, its, rel = krylov.gmres(A, lambda v: mf.apply_inverse(fh, v), b, rtol=1e-10)
    assert rel <= 1e-10 and its > 1
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_mf_hss_nonsymmetric_adjoint_identity():
    dims = (24, 24, 1)
    A = problems.grid_convdiff2d(24, 30.0, -20.0)
    A = A.to_scipy()
    fh = mf.factor(A, dims, mf.Options(hss_tol=1e-6, d0=64, dd=32, hss_min_front=64))
    rng = np.random.default_rng(9)
    b, c = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    lhs = c @ mf.apply_inverse(fh, b)
    rhs = mf.apply_inverse(fh, c, transpose=True) @ b
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


# -------------------------------------------------------------------- Krylov
def test_gmres_full_restart_is_exact():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((25, 25)) + 8 * np.eye(25)
    b = rng.standard_normal(25)
    x, its, rel = krylov.gmres(A, lambda v: v, b, rtol=1e-14, restart=30)
    assert its <= 25
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(x)


def test_gmres_restarted_monotone_and_exact_preconditioner():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((60, 60)) + 12 * np.eye(60)
    b = rng.standard_normal(60)
    x, its, rel = krylov.gmres(A, lambda v: v, b, rtol=1e-12, restart=5, maxit=500)
    assert rel <= 1e-12 and its > 5
    Ainv = np.linalg.inv(A)
    x, its, rel = krylov.gmres(A, lambda v: Ainv @ v, b, rtol=1e-12)
    assert its == 1
    x, its, rel = krylov.iterative_refinement(A, lambda v: Ainv @ v, b, rtol=1e-12)
    assert its <= 2


def test_dense_adjoint_matches_central_differences():
    """The oracle's adjoint gradient (dL/db, dL/dA on the pattern) equals
    central finite differences of L(x) = ||x - xt||^2 on a small
    nonsymmetric system."""
    from oracle import adjoint
    A = problems.grid_convdiff2d(5, 3.0, -2.0).to_scipy().tocsr()
    n = A.shape[0]
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, n)
    xt = rng.standard_normal(n)
    loss = lambda Am, bb: float(np.sum((np.linalg.solve(Am.toarray(), bb) - xt) ** 2))
    x, gb, gv = adjoint.dense_adjoint(A, b, lambda x: 2.0 * (x - xt))
    h = 1e-6
    for i in rng.choice(n, 5, replace=False):
        e = np.zeros(n); e[i] = h
        fd = (loss(A, b + e) - loss(A, b - e)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(fd))
    for p in rng.choice(A.nnz, 8, replace=False):
        Ap, Am = A.copy(), A.copy()
        Ap.data[p] += h; Am.data[p] -= h
        fd = (loss(Ap, b) - loss(Am, b)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-6 * max(1.0, abs(fd))


def test_anisotropic_grf_operator():
    """The variable-coefficient operator: symmetric positive definite;
    constant coefficient (sigma -> 0) gives the anisotropic 7-point Laplacian
    (faces 1, 1, 10); interior rows of any coefficient sum to zero; the
    random field has mean 0 and standard deviation sigma."""
    A = problems.grid_anisotropic_grf(6, sigma=1.0, seed=4).to_scipy()
    assert abs(A - A.T).max() == 0.0
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    c = problems.grid_anisotropic_grf(6, sigma=1e-14, seed=4).to_scipy().toarray()
    i = 1 + 6 * (1 + 6 * 1)  # interior cell (1, 1, 1)
    assert abs(c[i, i] - 24.0) < 1e-9
    assert abs(c[i, i - 1] + 1.0) < 1e-9 and abs(c[i, i - 6] + 1.0) < 1e-9 and abs(c[i, i - 36] + 10.0) < 1e-9
    interior = [x + 6 * (y + 6 * z) for x in range(1, 5) for y in range(1, 5) for z in range(1, 5)]
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.abs(rs[interior]).max() < 1e-12
    g = problems.gaussian_random_field(16, 4.0, 2.0, seed=9)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 2.0) < 1e-12


def test_batch_convdiff_generator():
    """The batch input: seeded sides in [lo, hi] and velocities in [-v, v],
    blocks equal to the single-system upwind operator, nothing between blocks,
    each block an M-matrix row pattern (positive diagonal dominating)."""
    sides, vel, A = problems.batch_convdiff2d(12, side_lo=5, side_hi=11, vmax=50.0, seed=3)
    sides2, vel2, A2 = problems.batch_convdiff2d(12, side_lo=5, side_hi=11, vmax=50.0, seed=3)
    assert sides == sides2 and np.array_equal(vel, vel2) and np.array_equal(A.values, A2.values)
    assert all(5 <= k <= 11 for k in sides) and np.all(np.abs(vel) <= 50.0)
    S = A.to_scipy().tocsr()
    off = 0
    for k, (vx, vy) in zip(sides, vel):
        n = k * k
        blk = S[off:off + n, off:off + n].toarray()
        ref = problems.grid_convdiff2d(k, vx, vy).to_scipy().toarray()
        assert np.array_equal(blk, ref)
        rest = S[off:off + n, :].toarray()
        rest[:, off:off + n] = 0.0
        assert not rest.any()
        assert np.all(np.diag(blk) >= np.abs(blk).sum(axis=1) - np.diag(blk) - 1e-9)
        off += n
    assert off == A.n


def _geometric_pattern_operator(n, radius, seed):
    from scipy.spatial import cKDTree
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    w = rng.uniform(0.5, 2.0, len(pairs))
    L = sp.csr_matrix((-np.concatenate([w, w]), (np.concatenate([pairs[:, 0], pairs[:, 1]]),
                                                  np.concatenate([pairs[:, 1], pairs[:, 0]]))), shape=(n, n))
    M = (L + sp.diags(-np.asarray(L.sum(axis=1)).ravel() + 0.05)).tocsr()
    M.sort_indices()
    return M


def test_algebraic_ordering_is_a_valid_elimination_structure():
    """Oracle algebraic nested dissection: a permutation; the subtrees of two
    sibling fronts share no edge; every I^upd contains the brute-force
    elimination's and lies after the separator; leaves of at most 64
    vertices; one root per connected component."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    M = _geometric_pattern_operator(600, 0.13, 4)
    M = sp.block_diag([M, problems.grid_poisson((7, 5, 1)).to_scipy()]).tocsr()  # two components
    n = M.shape[0]
    perm, fronts, Anew = ordering.analyze_csr(M)
    assert sorted(perm.tolist()) == list(range(n))
    ncomp = connected_components(M, directed=False)[0]
    assert sum(f.parent < 0 for f in fronts) == ncomp
    # brute-force elimination of the permuted pattern
    adj = [set(Anew.indices[Anew.indptr[i]:Anew.indptr[i + 1]].tolist()) - {i} for i in range(n)]
    for v in range(n):
        later = [w for w in adj[v] if w > v]
        for a in later:
            adj[a].update(w for w in later if w != a)
    for i, f in enumerate(fronts):
        bf = set()
        for v in range(f.sep_begin, f.sep_end):
            bf.update(w for w in adj[v] if w >= f.sep_end)
        assert bf <= set(f.upd.tolist()) and all(g >= f.sep_end for g in f.upd)
        if not f.children:
            assert f.ns <= 64
        if len(f.children) == 2:
            a, b = (fronts[c] for c in f.children)
            va = set(range(a.first, a.sep_end))
            vb = set(range(b.first, b.sep_end))
            for v in va:
                assert not (set(Anew.indices[Anew.indptr[v]:Anew.indptr[v + 1]].tolist()) & vb)


def test_factor_csr_is_exact_without_compression_and_as_eps_goes_to_zero():
    import scipy.sparse.linalg as spla
    M = _geometric_pattern_operator(900, 0.11, 6)
    b = problems.rhs_uniform(M.shape[0], 1, 2)[:, 0]
    xd = spla.spsolve(M.tocsc(), b)
    fz = mf.factor_csr(M, mf.Options())  # dense fronts only
    assert np.linalg.norm(mf.apply_inverse(fz, b) - xd) <= 1e-10 * np.linalg.norm(xd)
    fh = mf.factor_csr(M, mf.Options(hss_tol=1e-13, hss_min_front=64, d0=16, dd=16, hss_leaf=16))
    assert any(d is not None and hasattr(d, "H") for d in fh.data)
    assert np.linalg.norm(mf.apply_inverse(fh, b) - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(mf.apply_inverse(fh, b, transpose=True) - spla.spsolve(M.T.tocsc(), b)) \
        <= 1e-9 * np.linalg.norm(xd)


def test_caller_tree_is_validated_by_the_oracle():
    M = problems.grid_poisson((8, 8, 1)).to_scipy()
    n = M.shape[0]
    ident = np.arange(n)
    with pytest.raises(ValueError):
        ordering.analyze_csr(M, perm=ident, sep_ptr=[0, 32, n], parent=[-1, -1])  # not an elimination tree
    with pytest.raises(ValueError):
        ordering.analyze_csr(M, perm=ident, sep_ptr=[0, 16, 32, 48, n], parent=[3, 3, 3, -1])
    perm, fronts, _ = ordering.analyze_csr(M, perm=ident, sep_ptr=[0, n], parent=[-1])
    assert len(fronts) == 1 and fronts[0].nu == 0


def _path_pattern(n):
    rows = np.concatenate([np.arange(n - 1), np.arange(1, n), np.arange(n)])
    cols = np.concatenate([np.arange(1, n), np.arange(n - 1), np.arange(n)])
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))


def _fronts_as_lists(perm, fronts):
    """(separator vertices in natural numbering, children) per front."""
    return [(perm[f.sep_begin:f.sep_end].tolist(), list(f.children)) for f in fronts]


def test_algebraic_nd_path_of_40_worked_by_hand():
    """Path 0-1-...-39, leaves of at most 16 vertices (nd_leaf 4).  Worked by
    hand from the level-structure rule: the first search from vertex 0 ends
    at 39; the second search from 39 gives level(v) = 39 - v; levels 0..19
    hold 20 vertices and adding level 20 would pass half of 40, so level 20
    (vertex 19) is the separator, the near side is 39..20 (search order) and
    the far side 18..0.  The near side (20 vertices): searches from 39 then
    from 20, level(v) = v - 20, cumulative count passes 10 at level 10:
    separator 30, near 20..29, far 31..39 (leaves).  The far side (19
    vertices): level(v) = v from 0, passes 9.5 at level 9: separator 9, near
    0..8, far 10..18.  Postorder: near subtree, far subtree, separator."""
    perm, fronts, _ = ordering.analyze_csr(_path_pattern(40), nd_leaf=4, hss_leaf=8)
    want = [
        (list(range(20, 30)), []),
        (list(range(31, 40)), []),
        ([30], [0, 1]),
        (list(range(0, 9)), []),
        (list(range(10, 19)), []),
        ([9], [3, 4]),
        ([19], [2, 5]),
    ]
    assert _fronts_as_lists(perm, fronts) == want
    assert [f.parent for f in fronts] == [2, 2, 6, 5, 5, 6, -1]
    # I^upd in the new numbering: vertex 30 is new index 19, 9 is 38, 19 is 39
    assert [f.upd.tolist() for f in fronts] == [[19, 39], [19], [39], [38], [38, 39], [39], []]


def test_algebraic_nd_star_worked_by_hand():
    """Star: centre 0 joined to 1..40 (leaves of at most 16).  The second
    search starts at 40: level 0 = {40}, level 1 = {0}, level 2 = 1..39; the
    depth is 2, so the separator is level 1 (the centre), the near side {40}
    and the far side 1..39, which is disconnected.  A disconnected set splits
    its components (all single vertices, taken in order) between two groups,
    each to the group with fewer vertices so far (the first on a tie): odd
    vertices 1..39 and even vertices 2..38; the last vertex of the second
    group (38) is the separator.  The odd group (20 > 16) splits again into
    1, 5, ..., 37 and 3, 7, ..., 39 with separator 39; the even group without
    38 (18 > 16) into 2, 6, ..., 34 and 4, 8, ..., 36 with separator 36."""
    n = 41
    rows = np.concatenate([np.zeros(40, dtype=int), np.arange(1, 41), np.arange(n)])
    cols = np.concatenate([np.arange(1, 41), np.zeros(40, dtype=int), np.arange(n)])
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    perm, fronts, _ = ordering.analyze_csr(M, nd_leaf=4, hss_leaf=8)
    want = [
        ([40], []),
        (list(range(1, 38, 4)), []),
        (list(range(3, 36, 4)), []),
        ([39], [1, 2]),
        (list(range(2, 35, 4)), []),
        (list(range(4, 33, 4)), []),
        ([36], [4, 5]),
        ([38], [3, 6]),
        ([0], [0, 7]),
    ]
    assert _fronts_as_lists(perm, fronts) == want
