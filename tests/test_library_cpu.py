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
