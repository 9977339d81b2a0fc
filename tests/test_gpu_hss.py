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
