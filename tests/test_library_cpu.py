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
