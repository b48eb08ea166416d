"""Pins of the ILU(0) oracle and the library's host factorisation (CPU only).

The oracle (Saad, Algorithm 10.4) is pinned to what ILU(0) means, not to a
retyped copy of itself:
  * on a tridiagonal matrix the exact LU factors have no fill, so ILU(0) is
    the exact LU: L U = A;
  * with the full pattern ILU(0) is LU without pivoting, the textbook
    Doolittle factorisation: L U = A;
  * on any pattern, the defining property: (L U)_ij = A_ij for every (i, j)
    in the pattern (entries outside it are the dropped fill);
  * a dropped division or a wrong update order breaks the property.
The library's host routine (apcloud_ilu0_factor_host, the factorisation of the
comparison solve) must then match the oracle on random sparse patterns and
reject malformed input.
"""
import numpy as np
import pytest

from oracle.ilu import ilu0, packed


def _diag_dominant(rng, n, density):
    P = rng.random((n, n)) < density
    A = np.where(P, rng.normal(size=(n, n)), 0.0)
    np.fill_diagonal(A, np.abs(A).sum(axis=1) + 1.0 + rng.random(n))
    return A


def test_tridiagonal_is_exact_lu():
    rng = np.random.default_rng(1)
    n = 12
    A = np.diag(4.0 + rng.random(n)) + np.diag(rng.normal(size=n - 1), 1) + np.diag(rng.normal(size=n - 1), -1)
    L, U = ilu0(A)
    assert np.allclose(L @ U, A, rtol=0, atol=1e-14 * np.abs(A).max())


def test_full_pattern_is_lu_without_pivoting():
    rng = np.random.default_rng(2)
    A = _diag_dominant(rng, 9, 1.0)
    L, U = ilu0(A, pattern=np.ones_like(A, dtype=bool))
    assert np.allclose(L @ U, A, rtol=0, atol=1e-13 * np.abs(A).max())
    assert np.allclose(np.diag(L), 1.0) and np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.tril(U, -1), 0.0)


@pytest.mark.parametrize("seed,n,density", [(3, 20, 0.15), (4, 40, 0.08), (5, 30, 0.3)])
def test_product_matches_a_on_the_pattern(seed, n, density):
    rng = np.random.default_rng(seed)
    A = _diag_dominant(rng, n, density)
    P = (A != 0) | np.eye(n, dtype=bool)
    L, U = ilu0(A)
    LU = L @ U
    assert np.allclose(LU[P], A[P], rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.all(L[~P & ~np.eye(n, dtype=bool)] == 0.0) and np.all(U[~P] == 0.0)
    # with fill somewhere the incomplete factors are not the exact LU
    full_L, full_U = ilu0(A, pattern=np.ones_like(P))
    if not np.allclose(full_L @ full_U - LU, 0.0):
        assert np.abs(LU - A).max() > 0.0


def test_property_catches_a_dropped_division():
    rng = np.random.default_rng(6)
    A = _diag_dominant(rng, 15, 0.2)
    P = (A != 0) | np.eye(15, dtype=bool)
    a = A.copy()
    for i in range(1, 15):          # the IKJ loop without a_ik / a_kk
        for k in range(i):
            if P[i, k]:
                for j in range(k + 1, 15):
                    if P[i, j]:
                        a[i, j] -= a[i, k] * a[k, j]
    L, U = np.tril(a, -1) + np.eye(15), np.triu(a)
    assert not np.allclose((L @ U)[P], A[P], atol=1e-10)


def _csr(A):
    n = A.shape[0]
    P = (A != 0) | np.eye(n, dtype=bool)
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        js = np.nonzero(P[i])[0]
        cols.extend(js.tolist())
        vals.extend(A[i, js].tolist())
        rp[i + 1] = len(cols)
    return rp, np.array(cols, dtype=np.int32), np.array(vals), P


@pytest.mark.parametrize("seed,n,density", [(11, 50, 0.06), (12, 120, 0.03), (13, 60, 0.2)])
def test_library_host_factorisation_matches_oracle(seed, n, density):
    from paper_1603_04039_gb300 import ilu0_factor_host
    rng = np.random.default_rng(seed)
    A = _diag_dominant(rng, n, density)
    rp, cj, v, P = _csr(A)
    got = ilu0_factor_host(rp, cj, v)
    L, U = ilu0(A)
    want = packed(L, U, P)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-14 * np.abs(want).max())


def test_library_host_factorisation_rejects_bad_input():
    from paper_1603_04039_gb300 import APCloudError, ilu0_factor_host
    A = np.array([[4.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.0, 1.0, 4.0]])
    rp, cj, v, _ = _csr(A)
    bad = cj.copy()
    bad[[0, 1]] = bad[[1, 0]]                       # unsorted columns in row 0
    with pytest.raises(APCloudError):
        ilu0_factor_host(rp, bad, v)
    with pytest.raises(APCloudError):               # row 1 without its diagonal
        ilu0_factor_host(np.array([0, 2, 3, 5]), np.array([0, 1, 0, 1, 2], dtype=np.int32), np.ones(5))
    Z = np.array([[0.0, 1.0], [1.0, 1.0]])          # zero first pivot
    rpz, cjz, vz, _ = _csr(Z)
    with pytest.raises(APCloudError):
        ilu0_factor_host(rpz, cjz, vz)
