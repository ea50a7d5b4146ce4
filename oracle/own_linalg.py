"""The oracle's own dense linear algebra: Cholesky factorisation, triangular
solves, cyclic Jacobi for symmetric eigenproblems and one-sided (Hestenes)
Jacobi for the SVD, written out from their textbook definitions in FP64, and
the local steps of the preconditioner (Sec. 3.2 splitting, eq. (Zi)) built on
them instead of on LAPACK.

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it.  It shares no code
with the CUDA library.  Vector products of numpy are single steps; every
factorisation and rotation is spelled out here.

References for the algorithms (restated, not copied):
  * Cholesky: A = L L^T by rows (Cholesky-Banachiewicz), Golub & Van Loan,
    Matrix Computations, Sec. 4.2;
  * cyclic Jacobi for a symmetric matrix: rotations that zero one
    off-diagonal entry at a time in row-cyclic order, the rotation angle from
    the stable root of t^2 + 2 zeta t - 1 = 0 (Rutishauser), Golub & Van Loan
    Sec. 8.5;
  * one-sided Jacobi (Hestenes) for the SVD: rotations of pairs of rows until
    all rows are orthogonal; the row norms are the singular values and the
    normalised rows the right singular vectors, Golub & Van Loan Sec. 8.6.
"""
from __future__ import annotations

import numpy as np

U64 = 2.0 ** -53


def cholesky_lower(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with L L^T = A for symmetric positive definite A,
    row by row: L_jj = sqrt(A_jj - sum_k<j L_jk^2), then column j below the
    diagonal.  Raises ValueError at a pivot <= 0 (A not positive definite)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        piv = A[j, j] - L[j, :j] @ L[j, :j]
        if not piv > 0.0:
            raise ValueError(f"pivot {j} is {piv}: not positive definite")
        L[j, j] = np.sqrt(piv)
        if j + 1 < n:
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def solve_lower(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L X = B, forward substitution row by row."""
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    X = (B[:, None] if vec else B).copy()
    for i in range(L.shape[0]):
        X[i] = (X[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X[:, 0] if vec else X


def solve_upper_t(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L^T X = B (L lower triangular), backward substitution."""
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    X = (B[:, None] if vec else B).copy()
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X[:, 0] if vec else X


def _rotation(a: float, b: float, g: float):
    """c, s with [c -s; s c] making the pair with Gram [[a, g], [g, b]]
    orthogonal / the symmetric 2 x 2 block diagonal: t = tan(theta) is the
    smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / (2 g)."""
    zeta = (b - a) / (2.0 * g)
    t = np.copysign(1.0, zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, c * t, t


def jacobi_eigh(S: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """All eigenpairs of the symmetric S by cyclic Jacobi: each sweep visits
    the pairs (p, q), p < q, in row order and rotates rows and columns p, q so
    that the (p, q) entry vanishes; stop after a sweep in which every
    |S_pq| <= tol sqrt(|S_pp S_qq|).  Returns (w, V), eigenvalues ascending
    and orthonormal eigenvectors in the columns of V."""
    A = np.array(S, dtype=np.float64, copy=True)
    A = 0.5 * (A + A.T)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                g = A[p, q]
                if g == 0.0 or abs(g) <= tol * np.sqrt(abs(A[p, p] * A[q, q])):
                    continue
                rotated = True
                c, s, t = _rotation(A[p, p], A[q, q], g)
                # columns p, q then rows p, q: A <- J^T A J with J = I except
                # J_pp = J_qq = c, J_pq = s, J_qp = -s
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = A[q, p] = 0.0
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
        if not rotated:
            break
    else:
        raise RuntimeError("jacobi_eigh: sweep limit")
    w = np.diag(A).copy()
    o = np.argsort(w, kind="stable")
    return w[o], V[:, o]


def jacobi_svd_rows(X: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """One-sided Jacobi on the rows of X (m x n, m <= n): rotate pairs of rows
    (p, q) in row-cyclic order until every pair satisfies |<x_p, x_q>| <= tol
    ||x_p|| ||x_q||.  The rows are then sigma_j v_j^T.  Returns (sigma, Vt):
    singular values descending and the matching right singular vectors as
    rows (zero rows for zero singular values)."""
    Y = np.array(X, dtype=np.float64, copy=True)
    m = Y.shape[0]
    for _ in range(max_sweeps):
        rotated = False
        for p in range(m - 1):
            for q in range(p + 1, m):
                a = Y[p] @ Y[p]
                b = Y[q] @ Y[q]
                g = Y[p] @ Y[q]
                if g == 0.0 or abs(g) <= tol * np.sqrt(a * b):
                    continue
                rotated = True
                c, s, _ = _rotation(a, b, g)
                yp, yq = Y[p].copy(), Y[q].copy()
                Y[p] = c * yp - s * yq
                Y[q] = s * yp + c * yq
        if not rotated:
            break
    else:
        raise RuntimeError("jacobi_svd_rows: sweep limit")
    sig = np.sqrt(np.einsum("ij,ij->i", Y, Y))
    o = np.argsort(-sig, kind="stable")
    sig = sig[o]
    Vt = np.zeros_like(Y)
    nz = sig > 0.0
    Vt[nz] = Y[o][nz] / sig[nz, None]
    return sig, Vt


def orthonormal_complement(Vt: np.ndarray) -> np.ndarray:
    """Rows spanning the orthogonal complement of the row space of the
    orthonormal rows Vt (k x n): the unit vectors e_1 .. e_n are taken in turn,
    projected off the rows found so far twice (classical Gram-Schmidt applied
    twice), and kept when more than half of their norm survives.  Returns
    (n - k) x n orthonormal rows."""
    k, n = Vt.shape
    Q = [r for r in Vt]
    out = []
    for i in range(n):
        if len(Q) == n:
            break
        v = np.zeros(n)
        v[i] = 1.0
        for _ in range(2):
            B = np.array(Q)
            v = v - B.T @ (B @ v)
        nv = np.linalg.norm(v)
        if nv > 0.5:
            v = v / nv
            Q.append(v)
            out.append(v)
    if len(out) != n - k:
        raise RuntimeError("orthonormal_complement: rank")
    return np.array(out).reshape(n - k, n)


def splitting_root_own(X: np.ndarray, eps: float):
    """Sec. 3.2 with the own SVD: Abar_ii = V (Sigma + s1 eps I) V^T + s1 eps
    V_perp V_perp^T, V from one-sided Jacobi on the rows of X_i and V_perp its
    orthonormal complement.  Returns (Abar, sigma)."""
    sig, Vt = jacobi_svd_rows(X)
    Vp = orthonormal_complement(Vt)
    s1 = sig[0]
    Abar = (Vt.T * (sig + s1 * eps)) @ Vt + s1 * eps * (Vp.T @ Vp)
    return 0.5 * (Abar + Abar.T), sig


def local_eigenproblem_own(Aii: np.ndarray, Abar: np.ndarray, nI: int, tau: float):
    """Eq. (Zi) with the own factorisations, in the same reduction as the
    LAPACK oracle: S = Abar_II - Abar_IR Abar_RR^{-1} Abar_RI (R = [Gamma,
    Delta], Cholesky of Abar_RR), then the pencil S u = mu A_II u through the
    Cholesky factor L of A_II: C = L^{-1} S L^{-T}, cyclic Jacobi on C,
    u = L^{-T} w; lambda = 1/mu (mu <= 0 read as lambda = +inf).  Returns (lam,
    U_I, keep): lambda descending, the A_II-orthonormal eigenvectors on
    Omega_Ii, and the mask lambda > 1/tau."""
    BII, BIR, BRR = Abar[:nI, :nI], Abar[:nI, nI:], Abar[nI:, nI:]
    if BRR.shape[0]:
        LR = cholesky_lower(BRR)
        Y = solve_lower(LR, BIR.T)          # L_R^{-1} Abar_RI
        S = BII - Y.T @ Y
    else:
        S = BII.copy()
    S = 0.5 * (S + S.T)
    L = cholesky_lower(Aii[:nI, :nI])
    C = solve_lower(L, solve_lower(L, S).T)  # L^{-1} S L^{-T} (S symmetric)
    C = 0.5 * (C + C.T)
    mu, W = jacobi_eigh(C)
    uI = solve_upper_t(L, W)
    with np.errstate(divide="ignore"):
        lam = np.where(mu > 0.0, 1.0 / np.where(mu > 0.0, mu, 1.0), np.inf)
    return lam, uI, lam > 1.0 / tau
