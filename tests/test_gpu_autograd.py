"""Differentiation through the solver (torch.autograd): gradients of
L = ||x - xt||^2 with respect to b and to every stored entry of A, checked
against the oracle's dense-LU adjoint and against central differences, on
shifted Laplacians -Lap + sigma with sigma per cell uniform on [0, 10]."""
import numpy as np
import pytest

import problems
from oracle import adjoint

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problem(side, seed):
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(0.0, 10.0, side ** 3)
    A = problems.grid_shifted_laplacian3d(side, sigma)
    b = problems.rhs_uniform(A.n, 1, seed + 1)[:, 0]
    xt = np.random.default_rng(seed + 2).standard_normal(A.n)
    return A, b, xt


def _solver(A, side, **kw):
    import paper_1502_07405_gb300 as P
    s = P.Solver(P.Options.defaults(**kw))
    s.analyze_grid((side,) * 3, A.rowptr, A.colind)
    return s


def _grads(s, A, b, xt):
    from paper_1502_07405_gb300.autograd import sparse_solve
    vals = torch.tensor(A.values, device="cuda", requires_grad=True)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    x = sparse_solve(s, vals, bt)
    loss = ((x - torch.tensor(xt, device="cuda")) ** 2).sum()
    loss.backward()
    return x.detach().cpu().numpy(), bt.grad.cpu().numpy(), vals.grad.cpu().numpy(), float(loss.detach())


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_dense_adjoint_12cubed(prec):
    side = 12
    A, b, xt = _problem(side, 11)
    s = _solver(A, side, hss_tol=1e-6, hss_min_front=100, d0=32, dd=16, hss_leaf=32, precision=prec)
    x, gb, gv, _ = _grads(s, A, b, xt)
    assert s.get_stats()["n_hss_fronts"] > 0
    xo, gbo, gvo = adjoint.dense_adjoint(A.to_scipy().tocsr(), b, lambda x: 2.0 * (x - xt))
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    assert np.linalg.norm(gb - gbo) <= 1e-8 * np.linalg.norm(gbo)
    assert np.linalg.norm(gv - gvo) <= 1e-8 * np.linalg.norm(gvo)


def test_gradients_match_central_differences():
    side = 16
    A, b, xt = _problem(side, 21)
    s = _solver(A, side, hss_tol=1e-10, hss_min_front=256, d0=64, dd=32, rtol=1e-13, maxit=400)
    x, gb, gv, loss0 = _grads(s, A, b, xt)
    vals0 = torch.tensor(A.values, device="cuda")
    b0 = torch.tensor(b, device="cuda")
    xtt = torch.tensor(xt, device="cuda")

    def L(vals, bb):
        s.factor(vals)
        xx = s.solve(bb)
        return float(((xx - xtt) ** 2).sum())

    rng = np.random.default_rng(5)
    h = 1e-4  # (L is quadratic-like in the entries: O(h^2) truncation; the solves are exact to ~1e-13)
    for p in rng.choice(A.nnz, 6, replace=False):
        vp, vm = vals0.clone(), vals0.clone()
        vp[p] += h
        vm[p] -= h
        fd = (L(vp, b0) - L(vm, b0)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-4 * max(1.0, abs(fd)), (p, fd, gv[p])
    for i in rng.choice(A.n, 4, replace=False):
        bp, bm = b0.clone(), b0.clone()
        bp[i] += h
        bm[i] -= h
        fd = (L(vals0, bp) - L(vals0, bm)) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-4 * max(1.0, abs(fd)), (i, fd, gb[i])


def test_adjoint_identity_hss_24cubed():
    """<g, A^-1 b> = <A^-T g, b> with the compressed preconditioner (eps 1e-6,
    GMRES to 1e-10 both ways): the gradient path is the transposed solve."""
    side = 24
    A, b, xt = _problem(side, 31)
    s = _solver(A, side, hss_tol=1e-6, hss_min_front=512, d0=64, dd=32)
    x, gb, gv, _ = _grads(s, A, b, xt)
    assert s.get_stats()["n_hss_fronts"] > 0
    g = 2.0 * (x - xt)
    assert abs(np.dot(g, x) - np.dot(gb, b)) <= 1e-8 * abs(np.dot(g, x))
    # dL/dA on the pattern is -lambda_i x_j
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    np.testing.assert_allclose(gv, -gb[rows] * x[A.colind], rtol=1e-12, atol=1e-14)


def test_backward_after_refactor_raises():
    """The adjoint solve needs the factorization of the forward pass: if the
    same solver is factored again before backward, backward refuses instead
    of returning gradients of another matrix."""
    from paper_1502_07405_gb300.autograd import sparse_solve
    side = 8
    A, b, xt = _problem(side, 41)
    s = _solver(A, side, hss_min_front=1 << 30)
    vals = torch.tensor(A.values, device="cuda", requires_grad=True)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    loss = (sparse_solve(s, vals, bt) ** 2).sum()
    s.factor(torch.tensor(2.0 * A.values, device="cuda"))
    with pytest.raises(RuntimeError, match="factored again"):
        loss.backward()
    # a fresh forward pass on the current factorization differentiates normally
    vals2 = torch.tensor(A.values, device="cuda", requires_grad=True)
    (sparse_solve(s, vals2, bt) ** 2).sum().backward()
    assert torch.isfinite(vals2.grad).all()


def test_gradients_match_central_differences_48cubed_64_entries():
    """The 48^3 differentiation workload (shifted Laplacian, sigma ~ U[0, 10]
    per cell, HSS on fronts >= 1024 at eps 1e-6, L = ||x - xt||^2): the
    gradient with respect to 64 random stored entries of A (and 8 entries of
    b) against central differences.  The solves run GMRES to 1e-13 with the
    eps = 1e-6 preconditioner, so L carries a relative error near 1e-13 and
    the difference quotient a rounding error near 1e-13 L / h; h = 1e-4
    balances it against the O(h^2) truncation (h = 1e-6 would leave rounding
    errors of the order of the smaller gradient entries)."""
    side = 48
    A, b, xt = _problem(side, 51)
    s = _solver(A, side, hss_tol=1e-6, hss_min_front=1024, precision=1, rtol=1e-13, maxit=600)
    x, gb, gv, loss0 = _grads(s, A, b, xt)
    assert s.get_stats()["n_hss_fronts"] > 0
    vals0 = torch.tensor(A.values, device="cuda")
    b0 = torch.tensor(b, device="cuda")
    xtt = torch.tensor(xt, device="cuda")

    def L(vals, bb):
        s.factor(vals)
        xx = s.solve(bb)
        return float(((xx - xtt) ** 2).sum())

    h = 1e-4
    rng = np.random.default_rng(7)
    err = []
    for p in rng.choice(A.nnz, 64, replace=False):
        vp, vm = vals0.clone(), vals0.clone()
        vp[p] += h
        vm[p] -= h
        fd = (L(vp, b0) - L(vm, b0)) / (2 * h)
        err.append(abs(fd - gv[p]) / max(1.0, abs(fd)))
    for i in rng.choice(A.n, 8, replace=False):
        bp, bm = b0.clone(), b0.clone()
        bp[i] += h
        bm[i] -= h
        fd = (L(vals0, bp) - L(vals0, bm)) / (2 * h)
        err.append(abs(fd - gb[i]) / max(1.0, abs(fd)))
    assert max(err) <= 1e-3, max(err)
