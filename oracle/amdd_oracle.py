"""Plain, slow FP64 CPU oracle of the fully algebraic two-level overlapping
Schwarz preconditioner of Al Daas & Jolivet (arXiv 2109.05908).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library: it reads the same seeded inputs (module `synth`) and nothing else.

Every function follows the paper's definitions in the paper's order and
notation, with numpy / scipy (LAPACK) primitives as single steps (the module
own_linalg.py restates the SVD, Cholesky and symmetric eigensolver steps
without LAPACK, and the tests check the two against each other):

  Sec. 2.1      non-overlapping sets Omega_Ii, overlap Omega_Gi, extension
                Omega_Di, restrictions R_i, tilde R_i
  Eq. (Xi)      X_i = R_i A tilde R_i^T
  Sec. 3.2      economic SVD X_i = U S V^T, complement V_perp, regularised
                square root  Abar_ii = V (S + s1 eps I) V^T + s1 eps V_perp V_perp^T
  Eq. (tildeA)  tilde A_ii = X11 - X12 X22^{-1} X21 (Schur complement onto Omega_i)
  Eq. (Zi)      Z_i = span{u : D_i A_ii D_i u = lambda tilde A_ii u, lambda > 1/tau}
  Eq. (two_level_schwarz)
                M^{-1} = R_0^T (R_0 A R_0^T)^{-1} R_0 + sum_i R_i^T A_ii^{-1} R_i,
                R_0^T = [R_1^T D_1 Z_1, ..., R_N^T D_N Z_N]
  Sec. 1        preconditioned conjugate gradient (Hestenes-Stiefel), x0 = 0
  Sec. 4.1      the deflated form used in the experiments,
                M_deflated = R_0^T C_00^{-1} R_0 + M_RAS (I - A R_0^T C_00^{-1} R_0),
                M_RAS = sum_i R_i^T D_i A_ii^{-1} R_i (restricted additive
                Schwarz), inside right-preconditioned GMRES(m), x0 = 0

Readings where the paper is silent (each listed in the design notes):
  * overlap > 1: Omega_Gi = all nodes at graph distance 1..overlap from
    Omega_Ii, Omega_Di = the nodes at distance overlap+1;
  * D_i is Boolean: 1 on Omega_Ii, 0 on Omega_Gi;
  * eps = 2^-52 (double machine epsilon); the shift s1*eps*I is applied to the
    whole Abar_ii (Sec. 3.2 form of Remark 3.2);
  * the Boolean D_i makes D_i A_ii D_i singular on Omega_Gi; the zero
    eigenvalues (D_i u = 0) are never selected, and the non-zero part of the
    pencil is obtained by eliminating u on Omega_Gi from eq. (Zi) (textbook
    deflation of the kernel of D_i A_ii D_i, no approximation).  The
    eigenpairs are then those of the symmetric-definite pencil
    (S_i, A_II) with S_i the Schur complement of tilde A_ii onto Omega_Ii
    (= that of Abar_ii onto Omega_Ii, quotient property) and mu = 1/lambda;
  * stopping test ||r_k||_2 <= rtol ||b||_2 on the recursively updated
    residual, x0 = 0;
  * GMRES stops on the least-squares residual |g_{j+1}| <= rtol ||b||_2
    (equal to ||b - A x_j||_2 in exact arithmetic); the iteration count is
    the number of Arnoldi steps over all restart cycles.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS = 2.0 ** -52


def to_scipy(A) -> sp.csr_matrix:
    """CSR input (synth.CSR) as a scipy matrix."""
    return sp.csr_matrix((A.val, A.colind.astype(np.int64), A.rowptr), shape=(A.n, A.n))


# --------------------------------------------------------------------------
# Sec. 2.1: subdomains, overlap and extension layers
# --------------------------------------------------------------------------
def subdomain_sets(As: sp.csr_matrix, part: np.ndarray, i: int, overlap: int):
    """Omega_Ii (nodes with part == i), Omega_Gi (graph distance 1..overlap from
    Omega_Ii in G(A)) and Omega_Di (distance overlap+1), each ascending."""
    n = As.shape[0]
    dist = np.full(n, -1, dtype=np.int64)
    I = np.flatnonzero(part == i)
    dist[I] = 0
    frontier = I
    layers = []
    for d in range(1, overlap + 2):
        nb = np.unique(As[frontier].indices) if len(frontier) else np.zeros(0, np.int64)
        new = nb[dist[nb] < 0]
        dist[new] = d
        layers.append(np.sort(new))
        frontier = new
    G = np.sort(np.concatenate(layers[:overlap])) if overlap else np.zeros(0, np.int64)
    D = layers[overlap]
    return I, G, D


# --------------------------------------------------------------------------
# Eq. (Xi) and the local matrix A_ii
# --------------------------------------------------------------------------
def local_matrices(As: sp.csr_matrix, I, G, D):
    """A_ii = R_i A R_i^T and X_i = R_i A tilde R_i^T, with Omega_i = [I, G] and
    tilde Omega_i = [I, G, D] (concatenation order as in Sec. 2.1)."""
    om = np.concatenate([I, G])
    omt = np.concatenate([I, G, D])
    rows = As[om]
    X = rows[:, omt].toarray()
    Aii = rows[:, om].toarray()
    return Aii, X


# --------------------------------------------------------------------------
# Sec. 3.2: regularised square root of X_i^T X_i
# --------------------------------------------------------------------------
def splitting_root(X: np.ndarray, eps: float = EPS):
    """Abar_ii = V (Sigma + s1 eps I) V^T + s1 eps V_perp V_perp^T from the SVD
    of X_i (Sec. 3.2, Lemma 3.1 with the shift of Remark 3.2).  Returns
    (Abar, sigma) with sigma the singular values of X_i, descending."""
    n_i, nt = X.shape
    _, s, Vt = np.linalg.svd(X, full_matrices=True)
    V = Vt[:n_i].T           # economic right singular vectors (nt x n_i)
    Vp = Vt[n_i:].T          # orthonormal complement V_perp (nt x (nt - n_i))
    s1 = s[0]
    Abar = (V * (s + s1 * eps)) @ V.T + s1 * eps * (Vp @ Vp.T)
    return 0.5 * (Abar + Abar.T), s


def schur_overlap(Abar: np.ndarray, n_i: int) -> np.ndarray:
    """Eq. (tildeA): tilde A_ii = X11 - X12 X22^{-1} X21 with the (1,1) block on
    Omega_i and the (2,2) block on Omega_Di."""
    X11, X12 = Abar[:n_i, :n_i], Abar[:n_i, n_i:]
    X21, X22 = Abar[n_i:, :n_i], Abar[n_i:, n_i:]
    if X22.shape[0] == 0:
        return X11.copy()
    c = sla.cho_factor(X22, lower=True)
    T = X11 - X12 @ sla.cho_solve(c, X21)
    return 0.5 * (T + T.T)


# --------------------------------------------------------------------------
# Eq. (Zi): local generalized eigenproblem and selection
# --------------------------------------------------------------------------
def local_eigenproblem(Aii: np.ndarray, Abar: np.ndarray, nI: int, tau: float):
    """Eigenpairs of eq. (Zi), D_i A_ii D_i u = lambda tilde A_ii u, with D_i
    Boolean (1 on Omega_Ii, 0 on Omega_Gi).

    The kernel of D_i A_ii D_i (lambda = 0, u supported on Omega_Gi) is never
    selected.  Eliminating u_G from eq. (Zi) leaves A_II u_I = lambda S u_I
    with S the Schur complement of tilde A_ii onto Omega_Ii.  By the quotient
    property of Schur complements, S is also the Schur complement of Abar_ii
    onto Omega_Ii (eliminating Omega_Gi and Omega_Di at once), which is how it
    is formed here: S = Abar_II - Abar_IR Abar_RR^{-1} Abar_RI, R = [G, D].
    Abar_RR^{-1} is applied through its Cholesky factor (Abar_RR >= delta I
    with delta = s1 eps, the shift of Remark 3.2, so the factor exists).  The
    symmetric-definite pencil S u = mu A_II u is then solved with
    mu = 1/lambda.

    Returns (lam, U, keep): all nI non-zero eigenvalues lambda descending, the
    matching eigenvectors u on Omega_i (n_i x nI columns; the Omega_Ii part is
    A_II-orthonormal, the Omega_Gi part is the minimising extension) and the
    mask lambda > 1/tau."""
    n_i = Aii.shape[0]
    AII = Aii[:nI, :nI]
    BII, BIR, BRI, BRR = Abar[:nI, :nI], Abar[:nI, nI:], Abar[nI:, :nI], Abar[nI:, nI:]
    if BRR.shape[0]:
        c = sla.cho_factor(BRR, lower=True)
        S = BII - BIR @ sla.cho_solve(c, BRI)
    else:
        S = BII.copy()
    S = 0.5 * (S + S.T)
    mu, uI = sla.eigh(S, AII)            # ascending mu  <=>  descending lambda
    # S is positive definite in exact arithmetic (shifted splitting), so every
    # mu > 0; a mu <= 0 is rounding noise on an eps-cluster mode whose exact
    # lambda is ~1/(s1 eps) and is read as lambda = +inf.
    with np.errstate(divide="ignore"):
        lam = np.where(mu > 0.0, 1.0 / np.where(mu > 0.0, mu, 1.0), np.inf)
    U = np.zeros((n_i, nI))
    U[:nI] = uI
    if BRR.shape[0]:
        ext = -sla.cho_solve(c, BRI @ uI)
        U[nI:] = ext[: n_i - nI]
    keep = lam > 1.0 / tau
    return lam, U, keep


# --------------------------------------------------------------------------
# Setup of the two-level preconditioner
# --------------------------------------------------------------------------
@dataclass
class Subdomain:
    I: np.ndarray
    G: np.ndarray
    D: np.ndarray
    Aii: np.ndarray
    chol: tuple
    lam: np.ndarray       # all non-zero eigenvalues of eq. (Zi), descending
    keep: np.ndarray      # selection mask lambda > 1/tau
    Z: np.ndarray         # selected u (n_i x p_i)
    sigma: np.ndarray     # singular values of X_i

    @property
    def omega(self):
        return np.concatenate([self.I, self.G])

    @property
    def p(self):
        return int(self.keep.sum())


@dataclass
class Setup:
    A: sp.csr_matrix
    subs: list
    W: sp.csr_matrix            # R_0^T, n x n_C
    E: np.ndarray               # R_0 A R_0^T
    E_chol: tuple
    tau: float
    eps: float = EPS
    extra: dict = field(default_factory=dict)

    @property
    def nC(self):
        return self.W.shape[1]


def setup(A, part, N: int, overlap: int, tau: float, eps: float = EPS) -> Setup:
    """Setup in the paper's order: sets (Sec. 2.1), X_i (Eq. Xi), Abar_ii
    (Sec. 3.2), tilde A_ii (Eq. tildeA), local Cholesky of A_ii, local
    eigenproblem (Eq. Zi), coarse basis R_0^T = [R_i^T D_i Z_i] and
    coarse matrix R_0 A R_0^T with its Cholesky factor (Eq. two_level_schwarz)."""
    As = to_scipy(A) if not sp.issparse(A) else A.tocsr()
    n = As.shape[0]
    subs = []
    for i in range(N):
        I, G, D = subdomain_sets(As, part, i, overlap)
        Aii, X = local_matrices(As, I, G, D)
        Abar, s = splitting_root(X, eps)
        lam, U, keep = local_eigenproblem(Aii, Abar, len(I), tau)
        chol = sla.cho_factor(Aii, lower=True)
        subs.append(Subdomain(I, G, D, Aii, chol, lam, keep, U[:, keep], s))
    W = coarse_basis(subs, n)
    E = (W.T @ (As @ W)).toarray()
    E = 0.5 * (E + E.T)
    E_chol = sla.cho_factor(E, lower=True) if E.shape[0] else None
    return Setup(As, subs, W, E, E_chol, tau, eps)


def coarse_basis(subs, n: int) -> sp.csr_matrix:
    """R_0^T = [R_1^T D_1 Z_1, ..., R_N^T D_N Z_N]; with Boolean D_i the block
    of subdomain i is Z_i restricted to Omega_Ii rows."""
    rows, cols, vals = [], [], []
    off = 0
    for s in subs:
        nI = len(s.I)
        DZ = s.Z[:nI]                        # D_i Z_i (zero on Omega_Gi)
        r, c = np.nonzero(np.ones_like(DZ, dtype=bool))
        rows.append(s.I[r])
        cols.append(off + c)
        vals.append(DZ[r, c])
        off += s.p
    if off == 0:
        return sp.csr_matrix((n, 0))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, off))


# --------------------------------------------------------------------------
# Apply: Eq. (two_level_schwarz)
# --------------------------------------------------------------------------
def apply_one_level(S: Setup, r: np.ndarray) -> np.ndarray:
    """sum_i R_i^T A_ii^{-1} R_i r (one-level additive Schwarz)."""
    z = np.zeros_like(r)
    for s in S.subs:
        om = s.omega
        z[om] += sla.cho_solve(s.chol, r[om])
    return z


def apply_coarse(S: Setup, r: np.ndarray) -> np.ndarray:
    """R_0^T (R_0 A R_0^T)^{-1} R_0 r."""
    if S.nC == 0:
        return np.zeros_like(r)
    c = S.W.T @ r
    e = sla.cho_solve(S.E_chol, c)
    return S.W @ e


def apply(S: Setup, r: np.ndarray) -> np.ndarray:
    """z = M_additive^{-1} r (Eq. two_level_schwarz)."""
    return apply_coarse(S, r) + apply_one_level(S, r)


def apply_ras(S: Setup, r: np.ndarray) -> np.ndarray:
    """M_RAS r = sum_i R_i^T D_i A_ii^{-1} R_i r, the one-level restricted
    additive Schwarz method of Cai and Sarkis (Sec. 4.1).  With Boolean D_i
    every unknown takes the local solution of the one subdomain whose
    Omega_Ii holds it."""
    z = np.zeros_like(r)
    for s in S.subs:
        y = sla.cho_solve(s.chol, r[s.omega])
        z[s.I] += y[: len(s.I)]
    return z


def apply_deflated(S: Setup, r: np.ndarray) -> np.ndarray:
    """Sec. 4.1: M_deflated r = R_0^T C_00^{-1} R_0 r
    + M_RAS (r - A R_0^T C_00^{-1} R_0 r), C = A, C_00 = E."""
    zc = apply_coarse(S, r)
    return zc + apply_ras(S, r - S.A @ zc)


def gmres(As, b: np.ndarray, prec, restart: int = 30, rtol: float = 1e-8, maxit: int = 1000):
    """Right-preconditioned GMRES(m) (Saad and Schultz), x0 = 0: Arnoldi on
    A M with modified Gram-Schmidt, Givens rotations reducing the Hessenberg
    matrix, x = x0 + M V_j y_j at the end of each cycle.  Stops when the
    least-squares residual |g_{j+1}| <= rtol ||b||_2.  Returns (x, iterations,
    relative residual estimates, one per Arnoldi step)."""
    n = b.shape[0]
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [1.0 if nb else 0.0]
    if nb == 0.0:
        return x, 0, hist
    its = 0
    r = b.copy()
    while its < maxit:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((n, m + 1))
        Zp = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        done = False
        j = -1
        for j in range(m):
            Zp[:, j] = prec(V[:, j])
            w = As @ Zp[:, j]
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            hist.append(abs(g[j + 1]) / nb)
            if hist[-1] <= rtol or its >= maxit:
                done = True
                break
        k = j + 1
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + Zp[:, :k] @ y
        if done:
            break
        r = b - As @ x
    return x, its, hist


# --------------------------------------------------------------------------
# PCG
# --------------------------------------------------------------------------
def pcg(As, b: np.ndarray, prec, rtol: float = 1e-8, maxit: int = 1000, coeffs=None):
    """Preconditioned conjugate gradient (Hestenes-Stiefel), x0 = 0; stops when
    ||r_k||_2 <= rtol ||b||_2 (recursive residual).  Returns (x, iterations,
    relative residual history).  If `coeffs` is a list, the step lengths
    alpha_k and the ratios beta_k = (r_{k}, z_{k}) / (r_{k-1}, z_{k-1}) are
    appended to it as ("a", alpha) and ("b", beta) in the order computed."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb if nb else 0.0]
    if nb == 0.0:
        return x, 0, hist
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = As @ p
        alpha = rz / (p @ q)
        if coeffs is not None:
            coeffs.append(("a", alpha))
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            return x, k, hist
        z = prec(r)
        rz_new = r @ z
        if coeffs is not None:
            coeffs.append(("b", rz_new / rz))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def lanczos_extremes(coeffs):
    """Extreme eigenvalues of the Lanczos tridiagonal that k steps of PCG
    build implicitly (the CG-Lanczos relation, e.g. Saad, Iterative Methods
    for Sparse Linear Systems, Sec. 6.7.3): with step lengths alpha_j and
    ratios beta_j,
        T_11 = 1/alpha_1,  T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
        T_{j,j+1} = sqrt(beta_j)/alpha_j.
    Its eigenvalues are Ritz values of M^{-1} A, inside [lambda_min,
    lambda_max]; lambda_max(T)/lambda_min(T) is the condition estimate that
    the bound of Sec. 3.2 is checked against.  Returns (lambda_min,
    lambda_max), or (nan, nan) without a step."""
    al = [v for t, v in coeffs if t == "a"]
    be = [v for t, v in coeffs if t == "b"]
    k = len(al)
    if k == 0:
        return float("nan"), float("nan")
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def colouring_number(S) -> int:
    """k_c of Sec. 3.2: colours of a greedy colouring of the subdomain graph
    (i ~ j iff R_i A R_j^T != 0); any valid colouring gives a valid bound."""
    N = len(S.subs)
    A = S.A
    masks = []
    for s in S.subs:
        v = np.zeros(A.shape[0], dtype=bool)
        v[s.omega] = True
        masks.append(v)
    adj = np.zeros((N, N), dtype=bool)
    for i in range(N):
        reach = (abs(A) @ masks[i].astype(float)) > 0
        for j in range(N):
            adj[i, j] = i != j and bool((reach & masks[j]).any())
    col = -np.ones(N, dtype=int)
    for i in range(N):
        used = {col[j] for j in range(N) if adj[i, j] and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return int(col.max() + 1)


def splitting_constant(S) -> float:
    """k_m of Sec. 3.2: lambda_max(sum_i R_i^T tilde A_ii R_i, A) by a dense
    generalized eigenproblem (tiny inputs only)."""
    n = S.A.shape[0]
    Ad = S.A.toarray()
    T = np.zeros((n, n))
    for s in S.subs:
        Aii, X = local_matrices(S.A, s.I, s.G, s.D)
        Abar, _ = splitting_root(X, S.eps)
        T[np.ix_(s.omega, s.omega)] += schur_overlap(Abar, len(s.omega))
    return float(sla.eigh(T, Ad, eigvals_only=True).max())


def condition_bound(kc: int, km: float, tau: float) -> float:
    """Sec. 3.2: kappa(M^{-1} A) <= (k_c + 1)(2 + (2 k_c + 1) k_m / tau)."""
    return (kc + 1) * (2 + (2 * kc + 1) * km / tau)


def solve(A, part, N, overlap, tau, b, rtol=1e-8, maxit=1000):
    """Setup plus PCG with the two-level preconditioner."""
    S = setup(A, part, N, overlap, tau)
    x, its, hist = pcg(S.A, b, lambda r: apply(S, r), rtol, maxit)
    return S, x, its, hist
