"""FP64 CPU oracle of the learned eigensolver warm start (test infrastructure).

Only tests/, the smoke entry point and the benchmark's CPU baseline may import
this module; the library never does.

The local eigenproblem of eq. (Zi), reduced as in the method to the symmetric
T_i = L_A^{-1} S_i L_A^{-T} (eigenvalues mu = 1/lambda in [0, 1]), keeps the
p_i eigenvectors with mu < tau.  When the selection is partial those vectors
can be computed by an iterative block eigensolver started from an initial
block.  This module defines, as plain sequential code:

  * features(): 32 statistics of a subdomain's local matrix and sizes;
  * krylov_basis(): an orthonormal basis of the Krylov space
    K_16(A_II, 1) (classical Gram-Schmidt applied twice), the canonical
    "smooth" local basis on which proposals are expressed;
  * target_projector(): the projector onto the selected eigenvectors,
    expressed on that basis (16 x 16, invariant to the signs and rotations of
    the eigenvectors);
  * an MLP (32 -> 256 -> 256 -> 256, ReLU) whose 256 outputs, symmetrised as
    a 16 x 16 matrix, predict that projector; forward, backward (mean squared
    Frobenius error) and the Adam update (Kingma & Ba, 2015);
  * bf16(): round-to-nearest-even to bfloat16 (top 16 bits of binary32);
  * proposal(): the initial block from a predicted projector;
  * lobpcg(): block LOBPCG for the smallest eigenpairs of a symmetric matrix
    without preconditioner (Knyazev, SIAM J. Sci. Comput. 23 (2001)),
    Rayleigh-Ritz on span[X, R, P] with an orthonormalised trial basis.
"""
from __future__ import annotations

import numpy as np

NB = 16          # Krylov basis size
NF = 32          # features
NH = 256         # hidden width
NO = NB * NB     # outputs (a 16 x 16 matrix, symmetrised)


# --------------------------------------------------------------------- features
def _stats(v):
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        return [0.0, 0.0, 0.0, 0.0]
    return [float(v.mean()), float(v.std()), float(v.min()), float(v.max())]


def features(Aii: np.ndarray, nI: int, nG: int, nD: int, p: int, tau: float) -> np.ndarray:
    """32 statistics of subdomain i.  Aii is the dense local matrix ordered
    [Omega_I, Omega_Gamma]; A_II its leading nI x nI block, A_IG the coupling
    block.  Every entry is a symmetric function of the unknowns of Omega_I
    (invariant to their order)."""
    AII = Aii[:nI, :nI]
    AIG = Aii[:nI, nI:]
    d = np.diag(AII).copy()
    off = AII - np.diag(d)
    nz = off[off != 0.0]
    deg = (off != 0.0).sum(axis=1)
    cg = np.abs(AIG).sum(axis=1) / d
    dom = np.abs(off).sum(axis=1) / d
    ld = np.log(d)
    f = [np.log(nI), np.log1p(nG), np.log1p(nD), nG / nI, nD / nI]
    f += _stats(ld)
    f += _stats(np.log(np.abs(nz)))
    f += [f[8] - f[7]]
    f += [float(deg.mean()), float(deg.std()), float(deg.max())]
    f += [float((cg > 0).mean()), float(cg.mean()), float(cg.max())]
    f += _stats(dom)
    f += [np.log(np.linalg.norm(AII) / nI), np.log(d.sum() / nI)]
    f += [float((nz > 0).mean()) if nz.size else 0.0]
    f += [np.log(max(p, 1) / nI), np.log(max(p, 1))]
    f += [np.log(tau)]
    bnd = cg > 0
    f += [float(ld[bnd].mean() - ld.mean()) if bnd.any() else 0.0]
    f += [1.0]
    out = np.array(f, dtype=np.float64)
    assert out.shape == (NF,)
    return out


# --------------------------------------------------------------- local basis
def krylov_basis(AII: np.ndarray, k: int = NB) -> np.ndarray:
    """Orthonormal basis of K_k(A_II, 1): v_0 = 1 / sqrt(nI), then each new
    vector is A_II times the previous one, orthogonalised against all earlier
    vectors by classical Gram-Schmidt applied twice and normalised.  A vector
    whose norm falls below 1e-12 of its norm before orthogonalisation ends the
    space; the remaining columns are zero."""
    n = AII.shape[0]
    B = np.zeros((n, k))
    B[:, 0] = 1.0 / np.sqrt(n)
    for j in range(1, k):
        w = AII @ B[:, j - 1]
        w0 = np.linalg.norm(w)
        for _ in range(2):
            w = w - B[:, :j] @ (B[:, :j].T @ w)
        nw = np.linalg.norm(w)
        if not nw > 1e-12 * w0:
            break
        B[:, j] = w / nw
    return B


def target_projector(B: np.ndarray, U: np.ndarray) -> np.ndarray:
    """B^T Q Q^T B with Q an orthonormal basis of span(U) (U: the selected
    eigenvectors on Omega_I, one per column)."""
    Q, _ = np.linalg.qr(U)
    G = B.T @ Q
    return G @ G.T


# ---------------------------------------------------------------------- bf16
def bf16(x) -> np.ndarray:
    """Round binary32 values to bfloat16 (nearest, ties to even) and return
    them as float64: keep the top 16 bits of the binary32 encoding after adding
    0x7FFF plus the lowest kept bit."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


# ----------------------------------------------------------------------- MLP
def init_params(seed: int = 0) -> dict:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((NF, NH)) * np.sqrt(2.0 / NF), "b1": np.zeros(NH),
        "W2": rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH), "b2": np.zeros(NH),
        "W3": rng.standard_normal((NH, NO)) * np.sqrt(2.0 / NH), "b3": np.zeros(NO),
    }


def forward(P: dict, X: np.ndarray):
    """X: (batch, 32) standardised features.  Returns the symmetrised outputs
    (batch, 16, 16) and the activations needed by backward()."""
    z1 = X @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"] + P["b3"]
    Y = y.reshape(-1, NB, NB)
    Qh = 0.5 * (Y + Y.transpose(0, 2, 1))
    return Qh, (X, z1, h1, z2, h2)


def loss(Qh: np.ndarray, Qt: np.ndarray) -> float:
    """Mean over the batch of the squared Frobenius error."""
    return float(((Qh - Qt) ** 2).sum() / Qh.shape[0])


def backward(P: dict, Qh: np.ndarray, Qt: np.ndarray, cache) -> dict:
    """Gradient of loss() with respect to every parameter."""
    X, z1, h1, z2, h2 = cache
    nb = Qh.shape[0]
    dQ = 2.0 * (Qh - Qt) / nb
    dY = 0.5 * (dQ + dQ.transpose(0, 2, 1))  # through the symmetrisation
    dy = dY.reshape(nb, NO)
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = dy @ P["W3"].T
    dz2 = dh2 * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"].T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(P: dict, g: dict, state: dict, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (bias-corrected first and second moments)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in P:
        m = state.setdefault("m" + k, np.zeros_like(P[k]))
        v = state.setdefault("v" + k, np.zeros_like(P[k]))
        m *= b1
        m += (1 - b1) * g[k]
        v *= b2
        v += (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------ proposal
def proposal(Qh: np.ndarray, B: np.ndarray, m: int) -> np.ndarray:
    """The m leading eigenvectors of the predicted projector, mapped to
    Omega_I: B W (nI x m)."""
    w, V = np.linalg.eigh(0.5 * (Qh + Qh.T))
    W = V[:, ::-1][:, :m]
    return B @ W


# ------------------------------------------------------- reduced eigenproblem
def reduced_T(Aii: np.ndarray, Abar: np.ndarray, nI: int):
    """The symmetric matrix of eq. (Zi) in reduced form: S the Schur
    complement of Abar_ii onto Omega_Ii (Abar ordered [I, G, D] as the
    oracle's X_i columns), A_II = L_A L_A^T, T = L_A^{-1} S L_A^{-T}.  The
    eigenvalues of T are mu = 1/lambda and an eigenvector w of T gives
    u = L_A^{-T} w.  Returns (T, L_A)."""
    AII = Aii[:nI, :nI]
    BII, BIR, BRR = Abar[:nI, :nI], Abar[:nI, nI:], Abar[nI:, nI:]
    S = BII - BIR @ np.linalg.solve(BRR, BIR.T) if BRR.shape[0] else BII.copy()
    LA = np.linalg.cholesky(AII)
    Y = np.linalg.solve(LA, np.linalg.solve(LA, S).T)
    return 0.5 * (Y + Y.T), LA


# ------------------------------------------------------------------- LOBPCG
def _orth(S: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span(S): columns scaled to unit norm, then two
    passes of orthonormalisation through an eigendecomposition of the Gram
    matrix.  The first pass drops the directions with eigenvalue <= 1e-12 of
    the largest (above the rounding level of a Gram matrix, where the exact
    zeros of a rank-deficient S land); the second keeps eigenvalues > 1/2
    (the columns are then nearly orthonormal)."""
    nrm = np.linalg.norm(S, axis=0)
    S = S[:, nrm > 0] / nrm[nrm > 0]
    for it in range(2):
        G = S.T @ S
        w, V = np.linalg.eigh(0.5 * (G + G.T))
        keep = w > 1e-12 * max(w.max(), 1e-300) if it == 0 else w > 0.5
        S = S @ (V[:, keep] / np.sqrt(w[keep]))
    return S


def lobpcg(T: np.ndarray, X0: np.ndarray, p: int, tol: float = 1e-6, maxit: int = 200):
    """Block LOBPCG for the p smallest eigenpairs of the symmetric T, block
    size k = X0.shape[1] >= p.  Stops when every wanted residual
    ||T x_j - theta_j x_j|| <= tol (absolute; eigenvalues of T lie in [0, 1]).
    Returns (theta[:p], X[:, :p], iterations, converged)."""
    k = X0.shape[1]
    X = _orth(X0)
    TX = T @ X
    th, C = np.linalg.eigh(X.T @ TX)
    X, TX = X @ C, TX @ C
    P = None
    for it in range(maxit + 1):
        R = TX - X * th
        res = np.linalg.norm(R[:, :p], axis=0)
        if res.max() <= tol:
            return th[:p], X[:, :p], it, True
        if it == maxit:
            break
        blocks = [X, R] if P is None else [X, R, P]
        S = _orth(np.hstack(blocks))
        TS = T @ S
        G = S.T @ TS
        w, V = np.linalg.eigh(0.5 * (G + G.T))
        kk = min(k, S.shape[1])
        Cx = V[:, :kk]
        Xn = S @ Cx
        # search direction: the part of the new block outside the old X
        Pn = Xn - X @ (X.T @ Xn)
        X, TX, th = Xn, TS @ Cx, w[:kk]
        P = Pn
    return th[:p], X[:, :p], maxit, False
