"""Batches of independent grids (hssmf_analyze_grids): one elimination forest
whose levels are batched over every grid, R keyed by the row index inside its
grid, and refinement stopped per grid.  Upwinded 2D convection-diffusion
systems of uneven sizes, HSS on the larger fronts."""
import numpy as np
import pytest

import problems
from oracle import krylov, multifrontal as mf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRIDS = [(20, (3.0, -7.0)), (33, (-40.0, 12.0)), (48, (25.0, 49.0)), (64, (-10.0, -30.0)), (40, (0.5, -0.5))]
KW = dict(hss_tol=1e-6, hss_min_front=48, d0=16, dd=8, hss_leaf=16)  # 157 HSS fronts, 2-4 adaptive rounds


def _batch():
    mats = [problems.grid_convdiff2d(k, vx, vy) for k, (vx, vy) in GRIDS]
    return mats, problems.block_diag(mats)


def _solver(**kw):
    import paper_1502_07405_gb300 as P
    return P.Solver(P.Options.defaults(**kw))


def _batched(A, **kw):
    s = _solver(**kw)
    s.analyze_grids([(k, k, 1) for k, _ in GRIDS], A.rowptr, A.colind)
    s.factor(A.values)
    return s


def test_fp64_batched_application_equals_each_grid_alone_and_the_oracle():
    mats, A = _batch()
    s = _batched(A, maxit=0, precision=0, **KW)
    assert s.get_stats()["n_hss_fronts"] > 0
    b = problems.rhs_uniform(A.n, 2, 1)
    x = s.solve(b)
    off = 0
    for (k, _), m in zip(GRIDS, mats):
        bs = np.asfortranarray(b[off:off + m.n])
        t = _solver(maxit=0, precision=0, **KW)
        t.analyze_grid((k, k, 1), m.rowptr, m.colind)
        t.factor(m.values)
        xs = t.solve(bs)
        assert np.linalg.norm(x[off:off + m.n] - xs) <= 1e-13 * np.linalg.norm(xs)
        fo = mf.factor(m.to_scipy(), (k, k, 1), mf.Options(hss_tol=KW["hss_tol"], d0=KW["d0"], dd=KW["dd"],
                                                           hss_min_front=KW["hss_min_front"],
                                                           hss_leaf=KW["hss_leaf"]))
        xo = mf.apply_inverse(fo, bs)
        assert np.linalg.norm(xs - xo) <= 1e-9 * np.linalg.norm(xo)
        off += m.n


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_refinement_reaches_1e10_in_every_grid(prec):
    mats, A = _batch()
    s = _batched(A, precision=prec, **KW)
    b = problems.rhs_uniform(A.n, 3, 7)
    x = s.solve(b)
    st = s.get_stats()
    assert st["iterations"] >= 2  # eps = 1e-6 is not exact
    off = 0
    for m in mats:
        r = b[off:off + m.n] - m.to_scipy() @ x[off:off + m.n]
        rel = np.linalg.norm(r, axis=0) / np.linalg.norm(b[off:off + m.n], axis=0)
        assert np.all(rel <= 1e-10), rel
        off += m.n
    # device tensors, column-major view of a (nrhs, n) tensor
    bt = torch.tensor(np.ascontiguousarray(b.T), device="cuda").t()
    xt = s.solve(bt)
    assert np.allclose(xt.cpu().numpy(), x, rtol=0, atol=1e-12 * np.abs(x).max())


def test_batched_refinement_reports_nonconvergence():
    import paper_1502_07405_gb300 as P
    mats, A = _batch()
    s = _batched(A, precision=1, maxit=2, **dict(KW, hss_tol=1e-1))
    with pytest.raises(P.HssmfError) as e:
        s.solve(problems.rhs_uniform(A.n, 1, 1))
    assert e.value.status == P.ERR_NOCONV


def test_more_than_65535_fronts_in_one_level():
    """70000 independent 8 x 8 grids: level 0 holds 70000 fronts, above the
    65535 limit of a grid's y and z dimensions, so every per-front launch
    must index fronts along x.  Each grid is a scaled Poisson matrix (scale
    1 + grid index mod 7), dense fronts only: one application solves every
    grid to rounding and the refinement stops at once."""
    ng, side = 70000, 8
    base = problems.grid_poisson((side, side, 1))
    nb, zb = base.n, base.nnz
    scale = 1.0 + (np.arange(ng) % 7)
    rowptr = np.concatenate([[0], (base.rowptr[1:][None, :] + zb * np.arange(ng)[:, None]).ravel()])
    colind = (base.colind[None, :] + nb * np.arange(ng)[:, None]).ravel()
    values = (base.values[None, :] * scale[:, None]).ravel()
    A = problems.CSR(ng * nb, rowptr, colind, values)
    b = problems.rhs_uniform(A.n, 1, 3)
    s = _solver(precision=0)
    s.analyze_grids([(side, side, 1)] * ng, A.rowptr, A.colind)
    st = s.get_stats()
    assert st["n_fronts"] >= ng and st["n_hss_fronts"] == 0
    s.factor(A.values)
    x = s.solve(b)
    r = (b - A.to_scipy() @ x)[:, 0].reshape(ng, nb)
    rel = np.linalg.norm(r, axis=1) / np.linalg.norm(b[:, 0].reshape(ng, nb), axis=1)
    assert rel.max() <= 1e-12, rel.max()
    # the same grids solved one by one agree (spot check)
    for g in (0, 1, 65535, 65536, ng - 1):
        m = problems.grid_poisson((side, side, 1), scale=scale[g])
        xs = np.linalg.solve(m.to_scipy().toarray(), b[g * nb:(g + 1) * nb, 0])
        assert np.allclose(x[g * nb:(g + 1) * nb, 0], xs, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_dense_front_split_is_tuned_per_level_and_does_not_change_results(prec):
    """The autotuner times every distinct split of each level's dense fronts
    between the blocked panel path and the persistent shared-memory kernel
    and keeps the fastest; the persistent kernel repeats the panel path's
    operations in the same order, so every split gives the same solution
    bit for bit (here: tuned, untuned and a 3D grid whose largest fronts
    exceed the persistent kernel's bound)."""
    import paper_1502_07405_gb300 as P
    mats, A = _batch()
    b = problems.rhs_uniform(A.n, 3, 2)
    xs = []
    for tune in (True, False):
        s = _solver(maxit=0, precision=prec, **KW)
        s.set_autotune(tune)
        s.analyze_grids([(k, k, 1) for k, _ in GRIDS], A.rowptr, A.colind)
        s.factor(A.values)
        tun = s.get_tuning()
        F = P.Solver.TUNING_FIELDS
        assert tun.shape[1] == len(F) and tun.shape[0] == s.get_stats()["n_levels"]
        has_dense = tun[:, F.index("dense_fronts")] > 0
        assert (tun[has_dense, F.index("tuned")] == (1 if tune else 0)).all()
        assert (tun[:, F.index("panel_fronts")] <= tun[:, F.index("dense_fronts")]).all()
        xs.append(s.solve(b))
        s.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    dims = (20, 20, 20)  # 3D: the top fronts take the panel path in every split
    G = problems.grid_poisson(dims)
    bg = problems.rhs_uniform(G.n, 1, 3)
    out = []
    for tune in (True, False):
        s = _solver(maxit=0, precision=prec, hss_min_front=1 << 30)
        s.set_autotune(tune)
        s.analyze_grid(dims, G.rowptr, G.colind)
        s.factor(G.values)
        tun = s.get_tuning()
        assert tun[:, P.Solver.TUNING_FIELDS.index("panel_fronts")].max() > 0
        out.append(s.solve(bg))
        s.close()
    np.testing.assert_array_equal(out[0], out[1])
    xo = mf.apply_inverse(mf.factor(G.to_scipy(), dims, mf.Options()), bg)
    tol = 1e-10 if prec == 0 else 1e-4
    assert np.linalg.norm(out[0] - xo) <= tol * np.linalg.norm(xo)
