"""Pins of the symbolic Cholesky oracle (oracle/symbolic.py) against closed
forms and a numerical factorisation (CPU):
  * a path (tridiagonal) in natural order: no fill, parent k+1;
  * a star (arrow matrix): hub first fills everything (colcount n - k), hub
    last fills nothing;
  * the m x m five-point grid in natural order: every row past the first
    grid line fills its envelope, nnz(L) = 1 + 2 (m - 1) + (n - m)(m + 1),
    and the elimination tree is a chain;
  * random sparse SPD matrices: the non-zeros of numpy's Cholesky factor of
    P A P^T (random values, so no cancellation) are the predicted ones."""
import numpy as np

import synth
from oracle import symbolic as SY


def _csr(n, edges):
    rows = [i for i, j in edges] + [j for i, j in edges] + list(range(n))
    cols = [j for i, j in edges] + [i for i, j in edges] + list(range(n))
    A = synth._csr_from_coo(n, rows, cols, np.ones(len(rows)))
    return A.rowptr, A.colind


def test_path_has_no_fill():
    n = 9
    rp, ci = _csr(n, [(k, k + 1) for k in range(n - 1)])
    parent, cc = SY.eliminate(n, rp, ci, np.arange(n))
    assert np.array_equal(parent, np.r_[np.arange(1, n), -1])
    assert np.array_equal(cc, np.r_[np.full(n - 1, 2), 1])


def test_star_hub_first_and_last():
    n = 7
    rp, ci = _csr(n, [(0, k) for k in range(1, n)])
    _, cc = SY.eliminate(n, rp, ci, np.arange(n))
    assert np.array_equal(cc, n - np.arange(n))
    _, cc = SY.eliminate(n, rp, ci, np.r_[np.arange(1, n), 0])
    assert np.array_equal(cc, np.r_[np.full(n - 1, 2), 1])


def test_grid_natural_order_fills_the_row_envelopes():
    """A row i >= m of the factor fills its envelope [i - m, i] (through the
    previous grid line); a row 0 < i < m of the first line keeps only
    (i, i - 1).  So nnz(L) = 1 + 2 (m - 1) + (n - m)(m + 1), and the
    elimination tree is the chain k -> k + 1."""
    m = 6
    A = synth.laplace2d(m)
    n = A.n
    parent, cc = SY.eliminate(n, A.rowptr, A.colind, np.arange(n))
    assert cc.sum() == 1 + 2 * (m - 1) + (n - m) * (m + 1)
    assert np.array_equal(parent, np.r_[np.arange(1, n), -1])


def test_matches_numerical_cholesky():
    rng = np.random.default_rng(5)
    for n, p in ((30, 0.08), (40, 0.05), (25, 0.2)):
        B = (rng.uniform(size=(n, n)) < p)
        B = np.triu(B, 1)
        edges = list(zip(*np.nonzero(B)))
        rp, ci = _csr(n, edges)
        W = np.zeros((n, n))
        for i, j in edges:
            W[i, j] = W[j, i] = rng.uniform(-1, 1)
        M = W + np.diag(np.abs(W).sum(1) + 1.0)
        perm = rng.permutation(n)
        parent, cc = SY.eliminate(n, rp, ci, perm)
        L = np.linalg.cholesky(M[np.ix_(perm, perm)])
        nz = np.abs(L) > 0
        assert np.array_equal(nz.sum(0), cc)
        for k in range(n):
            below = np.flatnonzero(nz[k + 1:, k]) + k + 1
            assert parent[k] == (below[0] if len(below) else -1)
