"""Plain FP64 CPU oracle of the matrix-free form of the local eigensolve of
eq. (Zi) (Sec. 3.2, the paragraphs after eq. (Zi), eq. (invAii)).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

The paper solves eq. (Zi) with an iterative eigensolver that only needs
solves with tilde A_ii, and obtains them from the SVD of X_i without forming
the splitting: with X_i = U Sigma V^T (economic), eq. (invAii) gives

    Abar_ii^{-1} = V (Sigma + s1 eps I)^{-1} V^T + (s1 eps)^{-1} (I - V V^T).

With Boolean D_i, eq. (Zi) reduces to A_II u = lambda S u with S the Schur
complement of Abar_ii onto Omega_Ii (amdd_oracle.local_eigenproblem), and the
inverse of that Schur complement is the (I, I) block of Abar_ii^{-1} (block
inverse formula).  With A_II = L_A L_A^T the wanted eigenpairs are therefore
the LARGEST eigenpairs of the symmetric

    K = L_A^T (Abar_ii^{-1})_II L_A,      K y = lambda y,   u = L_A^{-T} y,

and A_II-orthonormal u follow from orthonormal y.  This module forms K
densely (the definition); the library reaches its largest eigenpairs
iteratively with K applied as four products, never forming Abar_ii, S or K.

Reading (listed in the design notes): the paper takes eps as the machine
precision.  In FP64 with eps = 2^-52 the two terms of eq. (invAii) cancel:
(I - V V^T) carries rounding of order 2^-53, which the factor (s1 eps)^{-1}
lifts to the size of the smallest terms of (Abar^{-1})_II.  The eigenvalues
near the threshold 1/tau then change by O(1) relative (pinned in
tests/test_matrix_free_oracle.py).  The matrix-free form is accurate only
when eps is far above the working precision; the library accepts it for
eps >= 2^-30 (errors about 2^-53 / eps relative).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import amdd_oracle as O


def inverse_splitting(X: np.ndarray, eps: float) -> np.ndarray:
    """Eq. (invAii): Abar_ii^{-1} from the economic SVD of X_i (columns in the
    order of X)."""
    _, s, Vt = np.linalg.svd(X, full_matrices=False)
    V = Vt.T
    d = s[0] * eps
    nt = X.shape[1]
    return (V / (s + d)) @ V.T + (np.eye(nt) - V @ V.T) / d


def operator(Aii: np.ndarray, X: np.ndarray, nI: int, eps: float) -> np.ndarray:
    """K = L_A^T (Abar_ii^{-1})_II L_A with the Omega_Ii unknowns first in the
    columns of X and in A_ii (the order of amdd_oracle.local_matrices)."""
    G = inverse_splitting(X, eps)[:nI, :nI]
    LA = np.linalg.cholesky(Aii[:nI, :nI])
    K = LA.T @ G @ LA
    return 0.5 * (K + K.T)


def local_eigs(Aii: np.ndarray, X: np.ndarray, nI: int, tau: float, eps: float):
    """All nI eigenvalues lambda of eq. (Zi) (descending) from K, the
    eigenvectors u = L_A^{-T} y (columns, A_II-orthonormal) and the mask
    lambda > 1/tau."""
    K = operator(Aii, X, nI, eps)
    lam, Y = np.linalg.eigh(K)
    lam, Y = lam[::-1], Y[:, ::-1]
    LA = np.linalg.cholesky(Aii[:nI, :nI])
    U = sla.solve_triangular(LA.T, Y, lower=False)
    return lam, U, lam > 1.0 / tau


def selection(A, part, N: int, overlap: int, tau: float, eps: float):
    """Per subdomain (lam, U_selected, p) of the matrix-free form."""
    As = O.to_scipy(A)
    out = []
    for i in range(N):
        I, G, D = O.subdomain_sets(As, np.asarray(part), i, overlap)
        Aii, X = O.local_matrices(As, I, G, D)
        lam, U, keep = local_eigs(Aii, X, len(I), tau, eps)
        out.append((lam, U[:, keep], int(keep.sum())))
    return out
