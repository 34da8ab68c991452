"""beta = 0 with an inactive box: the optimum of (pb_fe) is one linear KKT solve.

Without the L1 term and with bounds that never bind, (pb_fe) is an
equality-constrained QP whose first-order conditions are linear:
  [ M   0     L^T ] [y]   [ c_y ]
  [ 0   alpha M  -M ] [u] = [  0  ]
  [ L  -M     0   ] [p]   [  f  ]
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .qp import QP


def solve(qp: QP):
    n = qp.nI
    K = sp.bmat([[qp.Mcost, None, qp.L.T],
                 [None, qp.alpha * qp.M, -qp.M],
                 [qp.L, -qp.M, None]]).tocsc()
    rhs = np.concatenate([qp.cy, np.zeros(n), qp.fvec])
    x = spla.spsolve(K, rhs)
    return x[:n], x[n:2 * n], x[2 * n:]
