"""Pins of the oracle's deflated preconditioner, one-level restricted additive
Schwarz and right-preconditioned GMRES(m) (Sec. 4.1), against closed forms,
dense solves, brute-force least squares and the identities the definitions
imply (CPU)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import amdd_oracle as O


def _small_2d(m=12, box=4):
    A = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    return A, part, int(part.max()) + 1


def _small_3d(seed=1):
    A = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=seed, channel_value=1e3)
    part = synth.bfs_partition(A, 6, seed=seed, min_size=40, max_size=160)
    return A, part, int(part.max()) + 1


# ------------------------------------------------------------------ GMRES
def test_gmres_distinct_eigenvalues_closed_form():
    """With M = I and a diagonal A of k distinct values, the minimal
    polynomial has degree k: GMRES is exact at step k and not before."""
    rng = np.random.default_rng(0)
    k = 6
    d = np.repeat(np.arange(1.0, k + 1), 5)
    A = np.diag(d)
    b = rng.standard_normal(d.size)
    x, its, hist = O.gmres(A, b, lambda v: v, restart=20, rtol=1e-12)
    assert its == k
    assert hist[k - 1] > 1e-6
    assert np.allclose(x, b / d, atol=1e-12)


def test_gmres_matches_dense_solve_with_restarts():
    """Non-symmetric A and preconditioner, restart 7 (several cycles): the
    solution equals the dense solve."""
    rng = np.random.default_rng(1)
    n = 40
    A = rng.standard_normal((n, n)) + 8 * np.eye(n)
    Minv = np.linalg.inv(np.tril(A) + 0.5 * np.eye(n))
    b = rng.standard_normal(n)
    x, its, hist = O.gmres(A, b, lambda v: Minv @ v, restart=7, rtol=1e-12, maxit=400)
    assert its > 7 and hist[-1] <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10 * np.linalg.norm(np.linalg.solve(A, b)))


def test_gmres_minimal_residual_bruteforce():
    """Within one cycle step j minimises ||b - A M y|| over y in
    K_j(A M, b): its residual estimate equals the least-squares residual
    over an explicit Krylov basis."""
    rng = np.random.default_rng(2)
    n = 30
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    Minv = np.diag(1.0 / (np.abs(np.diag(A)) + 1.0))
    b = rng.standard_normal(n)
    _, _, hist = O.gmres(A, b, lambda v: Minv @ v, restart=30, rtol=1e-14, maxit=6)
    AM = A @ Minv
    for j in range(1, 6):
        K = np.column_stack([np.linalg.matrix_power(AM, i) @ b for i in range(j)])
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
        res = np.linalg.norm(b - AM @ Q @ y) / np.linalg.norm(b)
        assert np.isclose(hist[j], res, rtol=1e-8, atol=1e-14), (j, hist[j], res)


def test_gmres_zero_rhs():
    x, its, hist = O.gmres(np.eye(3), np.zeros(3), lambda v: v)
    assert its == 0 and np.all(x == 0)


# ------------------------------------------------------------------ RAS
def test_ras_single_subdomain_is_exact():
    """N = 1: M_RAS = A^{-1}."""
    m = 8
    A = synth.laplace2d(m)
    S = O.setup(A, np.zeros(m * m, dtype=np.int32), 1, 1, 0.5)
    x = synth.rhs(m * m, 4)
    assert np.allclose(O.apply_ras(S, S.A @ x), x, atol=1e-12)


def test_ras_without_overlap_is_block_jacobi():
    """Overlap 0: D_i = I on Omega_i = Omega_Ii, so M_RAS = M_ASM (block Jacobi)."""
    A, part, N = _small_2d()
    S = O.setup(A, part, N, 0, 0.5)
    r = synth.rhs(A.n, 1)
    assert np.array_equal(O.apply_ras(S, r), O.apply_one_level(S, r))


@pytest.mark.parametrize("maker", [_small_2d, _small_3d])
def test_ras_each_unknown_from_its_owner_dense(maker):
    """Each entry of M_RAS r is the entry of the dense local solve
    A[Omega_j, Omega_j]^{-1} r[Omega_j] of the subdomain j owning it, and on
    the overlap M_RAS differs from M_ASM."""
    A, part, N = maker()
    S = O.setup(A, part, N, 1, 0.5)
    Ad = S.A.toarray()
    r = synth.rhs(A.n, 2)
    z = O.apply_ras(S, r)
    for j in range(N):
        om = np.concatenate([np.flatnonzero(part == j), S.subs[j].G])
        y = np.linalg.solve(Ad[np.ix_(om, om)], r[om])
        own = part[om] == j
        assert np.allclose(z[om[own]], y[own], rtol=1e-10, atol=1e-12)
    assert np.abs(z - O.apply_one_level(S, r)).max() > 1e-3 * np.abs(z).max()


# ------------------------------------------------------------------ deflated
@pytest.mark.parametrize("maker,tau", [(_small_2d, 0.5), (_small_3d, 0.5), (_small_3d, 0.05)])
def test_deflated_fixes_the_coarse_range(maker, tau):
    """M_deflated A W = W + M_RAS (A W - A W E^{-1} W^T A W) = W, since
    E = W^T A W: the preconditioned operator is the identity on range(W)."""
    A, part, N = maker()
    S = O.setup(A, part, N, 1, tau)
    assert 0 < S.nC < A.n
    W = S.W.toarray()
    rng = np.random.default_rng(3)
    for c in rng.choice(S.nC, 8, replace=False):
        w = W[:, c]
        assert np.allclose(O.apply_deflated(S, S.A @ w), w, rtol=0, atol=1e-9 * np.abs(w).max())


def test_deflated_residual_is_orthogonal_to_the_coarse_space():
    """The deflated residual r - A W E^{-1} W^T r satisfies W^T(.) = 0."""
    A, part, N = _small_3d()
    S = O.setup(A, part, N, 1, 0.5)
    r = synth.rhs(A.n, 5)
    t = r - S.A @ O.apply_coarse(S, r)
    assert np.abs(S.W.T @ t).max() <= 1e-10 * np.abs(S.W.T @ r).max()


def test_deflated_exact_when_coarse_space_is_everything():
    """N = 1: the coarse space is R^n (every eigenvalue of eq. (Zi) is kept),
    W E^{-1} W^T = A^{-1}, the RAS term vanishes and GMRES takes one step."""
    m = 8
    A = synth.laplace2d(m)
    S = O.setup(A, np.zeros(m * m, dtype=np.int32), 1, 1, 50.0)
    assert S.nC == m * m
    b = synth.rhs(m * m, 6)
    x, its, hist = O.gmres(S.A, b, lambda r: O.apply_deflated(S, r), rtol=1e-10)
    assert its == 1
    assert np.allclose(x, np.linalg.solve(S.A.toarray(), b), atol=1e-10)


@pytest.mark.parametrize("maker", [_small_2d, _small_3d])
def test_deflated_gmres_converges_with_true_residual(maker):
    """GMRES(30) with M_deflated reaches 1e-8; its least-squares estimate is
    the true relative residual, and it takes fewer steps than with the
    one-level RAS alone."""
    A, part, N = maker()
    S = O.setup(A, part, N, 1, 0.5)
    b = synth.rhs(A.n, 7)
    x, its, hist = O.gmres(S.A, b, lambda r: O.apply_deflated(S, r), rtol=1e-8)
    true = np.linalg.norm(b - S.A @ x) / np.linalg.norm(b)
    assert hist[-1] <= 1e-8 and true <= 1e-8 and abs(true - hist[-1]) <= 1e-10
    _, its1, _ = O.gmres(S.A, b, lambda r: O.apply_ras(S, r), rtol=1e-8)
    assert its < its1


# ------------------------------------------------------------ planted mistakes
def test_planted_deflation_sign_is_caught(monkeypatch):
    """'+' instead of '-' in I - A W E^{-1} W^T breaks M_deflated A W = W."""
    def wrong(S, r):
        zc = O.apply_coarse(S, r)
        return zc + O.apply_ras(S, r + S.A @ zc)
    monkeypatch.setattr(O, "apply_deflated", wrong)
    with pytest.raises(AssertionError):
        test_deflated_fixes_the_coarse_range(_small_3d, 0.5)


def test_planted_ras_prolongation_is_caught(monkeypatch):
    """Prolongating the whole local solution (additive, no D_i) instead of its
    Omega_Ii part fails the owner-wise dense check."""
    monkeypatch.setattr(O, "apply_ras", O.apply_one_level)
    with pytest.raises(AssertionError):
        test_ras_each_unknown_from_its_owner_dense(_small_3d)


def test_planted_missing_rotation_is_caught(monkeypatch):
    """A GMRES that forgets to apply the earlier Givens rotations to the new
    Hessenberg column no longer solves the system."""
    def wrong(As, b, prec, restart=30, rtol=1e-8, maxit=1000):
        n = b.shape[0]
        x = np.zeros_like(b)
        r = b.copy()
        nb = np.linalg.norm(b)
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((n, m + 1))
        Zp = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        hist = [1.0]
        for j in range(m):
            Zp[:, j] = prec(V[:, j])
            w = As @ Zp[:, j]
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            hist.append(abs(g[j + 1]) / nb)
            if hist[-1] <= rtol:
                break
        k = j + 1
        x = Zp[:, :k] @ sla.solve_triangular(H[:k, :k], g[:k])
        return x, k, hist
    monkeypatch.setattr(O, "gmres", wrong)
    with pytest.raises(AssertionError):
        test_gmres_matches_dense_solve_with_restarts()
