"""GPU parity of the HSS-front path (sampling, Algorithm 1 with adaptive
rank, ULV, low-rank Schur update) against the FP64 CPU oracle."""
import numpy as np
import pytest

import problems
from oracle import krylov, multifrontal as mf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gpu(A, dims, **kw):
    import paper_1502_07405_gb300 as P
    s = P.Solver(P.Options.defaults(**kw))
    s.analyze_grid(dims, A.rowptr, A.colind)
    s.factor(A.values)
    return s


def _oracle(A, dims, **kw):
    o = mf.Options(hss_tol=kw.get("hss_tol", 1e-4), d0=kw.get("d0", 128), dd=kw.get("dd", 64),
                   hss_min_front=kw.get("hss_min_front", 1 << 30), hss_leaf=kw.get("hss_leaf", 128))
    return mf.factor(A.to_scipy(), dims, o)


def _relres(A, x, b):
    return np.linalg.norm(b - A.to_scipy() @ x, axis=0) / np.linalg.norm(b, axis=0)


HSS2D = dict(hss_min_front=64, d0=64, dd=32)


def test_tiny_eps_is_exact_2d():
    """eps -> 0: the HSS factorization is exact; one application matches the
    oracle's dense solution to 1e-10."""
    dims = (64, 64, 1)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 1)
    s = _gpu(A, dims, hss_tol=1e-14, maxit=0, **HSS2D)
    st = s.get_stats()
    assert st["n_hss_fronts"] > 20
    x = s.solve(b)
    xo = mf.apply_inverse(_oracle(A, dims), b)
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("eps", [1e-8, 1e-4])
def test_single_application_residual_within_10x_of_oracle_2d(eps):
    dims = (64, 64, 1)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 1)
    s = _gpu(A, dims, hss_tol=eps, maxit=0, **HSS2D)
    x = s.solve(b)
    fo = _oracle(A, dims, hss_tol=eps, **HSS2D)
    xo = mf.apply_inverse(fo, b)
    rg, ro = _relres(A, x, b)[0], _relres(A, xo, b)[0]
    assert rg <= 10 * ro + 1e-14, (rg, ro)
    # ranks agree up to pivot ties
    ro_max = max(r for _, _, r, _, _ in mf.hss_stats(fo))
    assert abs(s.get_stats()["max_rank"] - ro_max) <= max(2, ro_max // 10)


def test_gmres_to_1e10_3d_fp64_and_fp32():
    dims = (16, 16, 16)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 3, 1)
    for prec in (0, 1):
        s = _gpu(A, dims, hss_tol=1e-3, hss_min_front=256, d0=64, dd=32, precision=prec)
        x = s.solve(b)
        assert np.all(_relres(A, x, b) <= 1e-10)
        st = s.get_stats()
        assert st["n_hss_fronts"] > 0 and st["iterations"] >= 2


def test_3d_residual_within_10x_of_oracle():
    dims = (16, 16, 16)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 1)
    kw = dict(hss_tol=1e-2, hss_min_front=256, d0=64, dd=32, hss_leaf=32)
    s = _gpu(A, dims, maxit=0, **kw)
    x = s.solve(b)
    xo = mf.apply_inverse(_oracle(A, dims, **kw), b)
    rg, ro = _relres(A, x, b)[0], _relres(A, xo, b)[0]
    assert rg <= 10 * ro, (rg, ro)
    assert ro > 1e-8  # compression really is inexact here


def test_adaptive_rounds_grow_d():
    """d0 small: IDs fail, d grows by dd until they pass (Section 2.2.1)."""
    dims = (48, 48, 1)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 1)
    s = _gpu(A, dims, hss_tol=1e-12, hss_min_front=64, d0=16, dd=16, maxit=0)
    st = s.get_stats()
    assert st["adaptive_rounds"] > 0 and st["max_d"] > 16
    x = s.solve(b)
    assert _relres(A, x, b)[0] <= 1e-9


def _convdiff(side=64):
    return problems.grid_convdiff2d(side, 30.0, -20.0), (side, side, 1)


def test_solve_T_tiny_eps_is_exact_nonsymmetric_2d():
    """solve_T through HSS fronts: at eps -> 0 one application equals the
    oracle's transposed dense solution (A nonsymmetric) to 1e-10."""
    A, dims = _convdiff()
    b = problems.rhs_uniform(A.n, 2, 3)
    s = _gpu(A, dims, hss_tol=1e-14, maxit=0, **HSS2D)
    assert s.get_stats()["n_hss_fronts"] > 20
    x = s.solve_T(b)
    xo = mf.apply_inverse(_oracle(A, dims), b, transpose=True)
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
    r = b - A.to_scipy().T @ x
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_T_single_application_within_10x_of_oracle(prec):
    A, dims = _convdiff()
    b = problems.rhs_uniform(A.n, 1, 4)
    eps = 1e-6 if prec == 0 else 1e-4
    s = _gpu(A, dims, hss_tol=eps, maxit=0, precision=prec, **HSS2D)
    x = s.solve_T(b)
    fo = _oracle(A, dims, hss_tol=eps, **HSS2D)
    xo = mf.apply_inverse(fo, b, transpose=True)
    At = A.to_scipy().T
    rg = np.linalg.norm(b[:, 0] - At @ x[:, 0]) / np.linalg.norm(b)
    ro = np.linalg.norm(b[:, 0] - At @ xo[:, 0]) / np.linalg.norm(b)
    assert rg <= 10 * ro + (1e-14 if prec == 0 else 1e-6), (rg, ro)


def test_solve_and_solve_T_interleave():
    """solve_T builds the transposed ULV once; solve afterwards is unchanged."""
    A, dims = _convdiff()
    b = problems.rhs_uniform(A.n, 1, 5)
    s = _gpu(A, dims, hss_tol=1e-6, maxit=0, **HSS2D)
    x1 = s.solve(b)
    xt1 = s.solve_T(b)
    x2 = s.solve(b)
    xt2 = s.solve_T(b)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(xt1, xt2)
    assert np.linalg.norm(x1 - xt1) > 1e-6 * np.linalg.norm(x1)  # A is nonsymmetric


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_T_gmres_to_1e10(prec):
    A, dims = _convdiff()
    b = problems.rhs_uniform(A.n, 3, 6)
    s = _gpu(A, dims, hss_tol=1e-3, precision=prec, **HSS2D)
    x = s.solve_T(b)
    At = A.to_scipy().T
    rel = np.linalg.norm(b - At @ x, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(rel <= 1e-10), rel
    # and the 3D HSS path
    dims3 = (16, 16, 16)
    A3 = problems.grid_poisson(dims3)
    b3 = problems.rhs_uniform(A3.n, 2, 7)
    s3 = _gpu(A3, dims3, hss_tol=1e-3, hss_min_front=256, d0=64, dd=32, precision=prec)
    x3 = s3.solve_T(b3)
    assert np.all(_relres(A3, x3, b3) <= 1e-10)


@pytest.mark.parametrize("kind", ["poisson", "grf"])
def test_fp64_single_application_reproduces_oracle_3d(kind):
    """With the same seed, the FP64 form takes the oracle's decisions (ranks,
    skeletons, adaptive rounds) node by node, so one application of the
    compressed factorization (eps 1e-4, up to 3 adaptive rounds) agrees with
    the oracle's to rounding, not just in quality.  The FP32 form takes its own
    rounding-driven pivot choices: its residual is only held to 2x."""
    side = 20
    A = problems.grid_anisotropic_grf(side, 8.0, 1.0, (1.0, 1.0, 10.0), seed=0) if kind == "grf" \
        else problems.grid_poisson((side,) * 3)
    dims = (side,) * 3
    b = problems.rhs_uniform(A.n, 1, 1)
    kw = dict(hss_tol=1e-4, d0=64, dd=32, hss_min_front=256, hss_leaf=64)
    fo = _oracle(A, dims, **kw)
    xo = mf.apply_inverse(fo, b)
    ro = _relres(A, xo, b)[0]
    assert ro > 1e-5  # the compression is inexact at this tolerance
    s = _gpu(A, dims, maxit=0, precision=0, **kw)
    x = s.solve(b)
    assert s.get_stats()["n_hss_fronts"] == len(mf.hss_stats(fo))
    assert s.get_stats()["max_rank"] == max(r for _, _, r, _, _ in mf.hss_stats(fo))
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    s32 = _gpu(A, dims, maxit=0, precision=1, **kw)
    r32 = _relres(A, s32.solve(b), b)[0]
    assert r32 <= 2.0 * ro, (r32, ro)
