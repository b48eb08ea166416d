"""ILU(0) oracle -- TEST INFRASTRUCTURE ONLY (see the package docstring).

The incomplete LU factorisation with no fill outside a given pattern, in the
IKJ order of Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
Algorithm 10.4: for every row i, for every k < i in the pattern of row i
(increasing k), a_ik <- a_ik / a_kk, then a_ij <- a_ij - a_ik a_kj for every
j > k in the pattern of row i.  Dense arrays and plain loops, for small
matrices only.  It is the comparison baseline of the learned preconditioner;
the paper has no counterpart.
"""
from __future__ import annotations

import numpy as np


def ilu0(A, pattern=None):
    """A: dense (n, n) FP64 array.  pattern: boolean (n, n) array (default: the
    nonzeros of A plus the diagonal).  Returns (L, U): L unit lower triangular
    and U upper triangular, both zero outside the pattern."""
    a = np.array(A, dtype=np.float64)
    n = a.shape[0]
    P = (a != 0.0) if pattern is None else np.array(pattern, dtype=bool)
    P = P | np.eye(n, dtype=bool)
    a = np.where(P, a, 0.0)
    for i in range(1, n):
        for k in range(i):
            if not P[i, k]:
                continue
            a[i, k] = a[i, k] / a[k, k]
            for j in range(k + 1, n):
                if P[i, j]:
                    a[i, j] = a[i, j] - a[i, k] * a[k, j]
    L = np.tril(a, -1) + np.eye(n)
    U = np.triu(a)
    return L, U


def packed(L, U, pattern):
    """The factors packed like a CSR factorisation in place: L below the
    diagonal, U on and above it, read on the pattern (row-major order)."""
    M = np.tril(L, -1) + U
    return M[np.asarray(pattern, dtype=bool)]
