"""GPU parity of the dense multifrontal path (all fronts below the HSS
threshold) against the FP64 CPU oracle, through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import problems
from oracle import krylov, multifrontal as mf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    import paper_1502_07405_gb300 as P
    return P


def _solver(A, dims, **kw):
    P = _lib()
    kw.setdefault("hss_min_front", 1 << 30)
    s = P.Solver(P.Options.defaults(**kw))
    s.analyze_grid(dims, A.rowptr, A.colind)
    return s


def _oracle_x(A, dims, b, transpose=False):
    fz = mf.factor(A.to_scipy(), dims, mf.Options())
    return mf.apply_inverse(fz, b, transpose=transpose)


@pytest.mark.parametrize("nrhs", [2, 11])
@pytest.mark.parametrize("dims", [(64, 64, 1), (8, 8, 1), (33, 17, 1), (9, 7, 5), (16, 16, 16)])
def test_direct_solve_matches_oracle(dims, nrhs):
    """maxit = 0: one forward + backward sweep; uncompressed FP64 agrees with
    the oracle to relative error 1e-10 (elementwise over all n).  11 columns:
    the warp-per-column sweeps (two CTAs of 8 columns, the second ragged)."""
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, nrhs, 1)
    s = _solver(A, dims, maxit=0)
    s.factor(A.values)
    x = s.solve(b)
    xo = _oracle_x(A, dims, b)
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
    xt = s.solve_T(b)
    assert np.linalg.norm(xt - xo) <= 1e-10 * np.linalg.norm(xo)


def test_device_buffers_and_refinement_to_1e10():
    dims = (64, 64, 1)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 1, 1)[:, 0]
    s = _solver(A, dims)
    vals = torch.tensor(A.values, device="cuda")
    s.factor(vals)
    bt = torch.tensor(b, device="cuda")
    xt = s.solve(bt)
    torch.cuda.synchronize()
    x = xt.cpu().numpy()
    r = b - A.to_scipy() @ x
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    st = s.get_stats()
    assert st["relres"] <= 1e-10 and st["iterations"] >= 1 and st["n_hss_fronts"] == 0


def _nonsym(dims, seed):
    A = problems.grid_poisson(dims)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1, 1, A.nnz)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = rows == A.colind
    v[diag] = rng.uniform(0.2, 1.0, diag.sum()) * rng.choice([-1, 1], diag.sum())
    return problems.CSR(A.n, A.rowptr, A.colind, v)


@pytest.mark.parametrize("nrhs", [3, 11])
@pytest.mark.parametrize("dims", [(12, 12, 1), (6, 5, 4)])
def test_pivoting_nonsymmetric(dims, nrhs):
    A = _nonsym(dims, 3)
    b = problems.rhs_uniform(A.n, nrhs, 2)
    s = _solver(A, dims, maxit=0)
    s.factor(A.values)
    x = s.solve(b)
    xo = _oracle_x(A, dims, b)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    xt = s.solve_T(b)
    xto = _oracle_x(A, dims, b, transpose=True)
    assert np.linalg.norm(xt - xto) <= 1e-9 * np.linalg.norm(xto)


def test_fp32_factor_with_fp64_refinement():
    dims = (48, 48, 1)
    A = problems.grid_poisson(dims)
    b = problems.rhs_uniform(A.n, 4, 1)
    s = _solver(A, dims, precision=1)
    s.factor(A.values)
    x = s.solve(b)
    R = b - A.to_scipy() @ x
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-10 * np.linalg.norm(b, axis=0))
    assert s.get_stats()["iterations"] >= 2


def test_singular_matrix_reports_error():
    P = _lib()
    dims = (8, 8, 1)
    A = problems.grid_poisson(dims)
    s = _solver(A, dims)
    with pytest.raises(P.HssmfError) as e:
        s.factor(np.zeros(A.nnz))
    assert e.value.status == P.ERR_SINGULAR
    s.factor(A.values)  # the context stays usable
    x = s.solve(np.ones(A.n))
    assert np.linalg.norm(A.to_scipy() @ x - 1.0) <= 1e-10 * np.sqrt(A.n)
