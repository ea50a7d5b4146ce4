"""Plain CPU oracle of the symbolic Cholesky factorisation of a local matrix
in a given elimination order: the structure a sparse local factor (in place
of the exact dense Cholesky of A_ii, Sec. 4.1) would have.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

Graph elimination (the textbook definition): eliminating unknown k joins all
its not-yet-eliminated neighbours into a clique.  With the unknowns
renumbered so that perm[k] is eliminated k-th,
  * L(i, k) != 0 for i > k exactly when i is a neighbour of k at the time k
    is eliminated (no numerical cancellation assumed);
  * colcount[k] = 1 + the number of such i (the diagonal included);
  * parent[k] = the smallest such i (the elimination tree), -1 if none.
Dense boolean arithmetic, so for small n only.
"""
from __future__ import annotations

import numpy as np


def pattern(n: int, rowptr, colind) -> np.ndarray:
    """Symmetric boolean adjacency (no diagonal) of a CSR pattern."""
    G = np.zeros((n, n), dtype=bool)
    rowptr = np.asarray(rowptr)
    colind = np.asarray(colind)
    for r in range(n):
        G[r, colind[rowptr[r]:rowptr[r + 1]]] = True
    G = G | G.T
    np.fill_diagonal(G, False)
    return G


def eliminate(n: int, rowptr, colind, perm):
    """(parent, colcount) of the Cholesky factor of P A P^T, P the
    permutation with row k of P A P^T = row perm[k] of A."""
    perm = np.asarray(perm)
    G = pattern(n, rowptr, colind)[np.ix_(perm, perm)]
    parent = np.full(n, -1, dtype=np.int64)
    colcount = np.ones(n, dtype=np.int64)
    for k in range(n):
        nb = np.flatnonzero(G[k, k + 1:]) + k + 1
        colcount[k] += len(nb)
        if len(nb):
            parent[k] = nb[0]
            G[np.ix_(nb, nb)] = True
    np.fill_diagonal(G, False)
    return parent, colcount
