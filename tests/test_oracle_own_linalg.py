"""Pins of the oracle's own dense linear algebra (oracle/own_linalg.py) and the
cross-check of the LAPACK-based oracle steps against it.

Pins that do not come from the routines themselves:
  * Cholesky of tridiag(-1, 2, -1): the pivots are d_k = (k + 1)/k (closed form
    of the LDL^T recurrence d_k = 2 - 1/d_{k-1}), so L_kk = sqrt((k + 1)/k) and
    L_{k+1,k} = -sqrt(k/(k + 1)) (1-based k);
  * cyclic Jacobi on the 1D and 2D Dirichlet Laplacians: the closed-form
    spectra 2 - 2 cos(j pi/(n + 1)) and their sums over two directions;
  * one-sided Jacobi SVD of U diag(s) V^T with prescribed s: recovers s;
  * an indefinite matrix is refused at its first non-positive pivot;
  * a planted mistake (the rotation's sign flipped) is caught by the spectrum pin.
Then the Sec. 3.2 splitting and eq. (Zi) computed with these routines equal the
LAPACK oracle's on small Laplacian and channelled-diffusion subdomains.
"""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import own_linalg as L


def test_cholesky_closed_form_on_the_1d_laplacian():
    n = 12
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    Lf = L.cholesky_lower(T)
    k = np.arange(1, n + 1, dtype=float)
    assert np.allclose(np.diag(Lf), np.sqrt((k + 1) / k), rtol=0, atol=1e-15)
    assert np.allclose(np.diag(Lf, -1), -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=0, atol=1e-15)
    assert np.abs(np.triu(Lf, 1)).max() == 0.0


def test_cholesky_and_triangular_solves_on_random_spd():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((30, 30))
    A = M @ M.T + 30 * np.eye(30)
    Lf = L.cholesky_lower(A)
    assert np.abs(Lf @ Lf.T - A).max() <= 1e-13 * np.abs(A).max()
    b = rng.standard_normal((30, 3))
    x = L.solve_upper_t(Lf, L.solve_lower(Lf, b))
    assert np.abs(A @ x - b).max() <= 1e-12 * np.abs(b).max()
    with pytest.raises(ValueError):
        L.cholesky_lower(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_jacobi_eigh_closed_form_spectra():
    n = 15
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = L.jacobi_eigh(T)
    exact = np.sort(2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    assert np.abs(w - exact).max() <= 1e-14
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-14
    assert np.abs(T @ V - V * w).max() <= 1e-13
    m = 6  # 2D 5-point Laplacian on m x m: sums of two 1D spectra
    A = synth.laplace2d(m)
    D = np.zeros((A.n, A.n))
    for r in range(A.n):
        D[r, A.colind[A.rowptr[r]:A.rowptr[r + 1]]] = A.val[A.rowptr[r]:A.rowptr[r + 1]]
    w2, _ = L.jacobi_eigh(D)
    e1 = 2.0 - 2.0 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1))
    assert np.abs(w2 - np.sort((e1[:, None] + e1[None, :]).ravel())).max() <= 1e-13


def test_jacobi_svd_recovers_prescribed_singular_values():
    rng = np.random.default_rng(1)
    m, n = 9, 14
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.array([7.0, 5.0, 3.0, 2.0, 1.0, 0.5, 1e-3, 1e-6, 1e-9])
    X = (U * s) @ V[:, :m].T
    sig, Vt = L.jacobi_svd_rows(X)
    assert np.abs(sig - s).max() <= 1e-14 * s[0]
    assert np.abs(Vt @ Vt.T - np.eye(m)).max() <= 1e-12
    # the rows span the row space of X; the direction of singular value s_j
    # is fixed by X (itself rounded at u s_1) only to about u s_1 / s_j
    P = Vt.T @ Vt
    dev = np.abs(P @ V[:, :m] - V[:, :m]).max(axis=0)
    assert np.all(dev <= 1e-12 + 1e-14 * s[0] / s), dev
    Vp = L.orthonormal_complement(Vt)
    assert Vp.shape == (n - m, n)
    assert np.abs(Vp @ Vt.T).max() <= 1e-14
    assert np.abs(Vp @ Vp.T - np.eye(n - m)).max() <= 1e-14


def test_planted_rotation_sign_is_caught(monkeypatch):
    """The rotation with its sign flipped no longer zeroes the visited entry:
    the iteration stalls or misses the closed-form spectrum."""
    good = L._rotation

    def bad(a, b, g):
        c, s, t = good(a, b, g)
        return c, -s, -t

    monkeypatch.setattr(L, "_rotation", bad)
    n = 8
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    exact = np.sort(2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    try:
        w, _ = L.jacobi_eigh(T, max_sweeps=30)
    except RuntimeError:
        return
    assert np.abs(w - exact).max() > 1e-6


def _cases():
    A = synth.laplace2d(8)
    yield "lap8_box4", O.to_scipy(A), synth.box_partition_2d(8, 4), 1
    D = synth.diffusion3d(6, sigma=1.0, corr=2.0, n_channels=2, seed=3, channel_value=1e3)
    yield "diff6_bfs", O.to_scipy(D), synth.bfs_partition(D, 4, seed=3, min_size=30, max_size=90), 1


@pytest.mark.parametrize("eps", [2.0 ** -23, 2.0 ** -40])
def test_oracle_local_steps_match_the_own_routines(eps):
    """Singular values of X_i, the eigenvalues of eq. (Zi) (as mu = 1/lambda),
    the selection and the selected span, own routines against LAPACK."""
    for name, As, part, ov in _cases():
        N = int(part.max()) + 1
        for i in range(N):
            I, G, D = O.subdomain_sets(As, part, i, ov)
            Aii, X = O.local_matrices(As, I, G, D)
            Ab, s = O.splitting_root(X, eps)
            Ab2, s2 = L.splitting_root_own(X, eps)
            assert np.abs(s2 - s).max() <= 1e-13 * s[0], (name, i)
            assert np.abs(Ab2 - Ab).max() <= 1e-12 * s[0], (name, i)
            for tau in (0.5, 100.0):
                lam, U, keep = O.local_eigenproblem(Aii, Ab, len(I), tau)
                lam2, uI2, keep2 = L.local_eigenproblem_own(Aii, Ab2, len(I), tau)
                mu, mu2 = 1.0 / np.sort(lam), 1.0 / np.sort(lam2)
                assert np.abs(mu2 - mu).max() <= 1e-8 * mu.max() + 1e-9, (name, i, tau)
                assert keep2.sum() == keep.sum(), (name, i, tau)
                p = int(keep.sum())
                if 0 < p < len(I):
                    # selected spans: A_II-orthonormal bases, compare the projectors
                    AII = Aii[: len(I), : len(I)]
                    Z1 = U[: len(I), np.argsort(-lam)[:p]]
                    Z2 = uI2[:, np.argsort(-lam2)[:p]]
                    P1 = Z1 @ Z1.T @ AII
                    P2 = Z2 @ Z2.T @ AII
                    assert np.abs(P1 - P2).max() <= 1e-7, (name, i, tau)
