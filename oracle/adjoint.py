"""Oracle (test infrastructure only: imported by tests, never by the
library): the gradient of a loss through a sparse linear solve, by dense LU.

For x = A^-1 b and L(x), with g = dL/dx and lambda = A^-T g (standard
adjoint of a linear system; the differentiation interface of the solver,
not a result of the paper):

    dL/db = lambda,   dL/dA_ij = -lambda_i x_j  (on the stored entries).

Pinned in tests/test_oracle_pins.py by central finite differences of L.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def dense_adjoint(A, b, dLdx):
    """(x, dL/db, dL/dvalues) for a scipy CSR matrix A (values in CSR order),
    b (n,) and the function dLdx(x) -> (n,) upstream gradient."""
    Ad = A.toarray()
    lu = sla.lu_factor(Ad)
    x = sla.lu_solve(lu, b)
    g = dLdx(x)
    lam = sla.lu_solve(lu, g, trans=1)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    gvals = -lam[rows] * x[A.indices]
    return x, lam, gvals
