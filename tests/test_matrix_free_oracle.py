"""Pins of the oracle's matrix-free local eigensolve (Sec. 3.2, eq. (invAii);
oracle/matrix_free.py) against what the paper and the mathematics fix (CPU):

  * eq. (invAii) is the inverse of the regularised square root
    (X_i^T X_i)^{1/2} + s1 eps I, the latter built from an eigendecomposition
    of X_i^T X_i (a different library routine from the SVD the oracle uses);
  * the largest eigenvalues of K = L_A^T (Abar^{-1})_II L_A are those of the
    Schur-complement form of eq. (Zi) (amdd_oracle.local_eigenproblem: a
    Cholesky of the extension block instead of the SVD), with the same
    selection and the same selected span;
  * closed form: with no overlap and no extension (uncoupled blocks) X_i =
    A_ii, the splitting is A_ii + s1 eps I and lambda_j = a_j / (a_j + s1 eps)
    for the eigenvalues a_j of A_ii (a large eps makes the selection partial);
  * at eps = 2^-52 the two terms of eq. (invAii) cancel in FP64 and the
    eigenvalues near 1/tau move by O(1) relative: the reason the library
    takes the matrix-free form only for eps >= 2^-30."""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import matrix_free as MF

EPS23 = 2.0 ** -23


def _cases():
    M = synth.diffusion3d(10, sigma=1.0, corr=2.0, n_channels=2, seed=2, channel_value=1e3)
    part = synth.bfs_partition(M, 10, seed=2, min_size=50, max_size=180)
    yield "diff10_bfs", M, part, int(part.max()) + 1, 1, 0.5
    M = synth.laplace2d(24)
    yield "lap24_box6", M, synth.box_partition_2d(24, 6), 16, 1, 0.5
    yield "lap24_box6_ov2", M, synth.box_partition_2d(24, 6), 16, 2, 0.7


CASES = {c[0]: c[1:] for c in _cases()}


def _local(M, part, i, ov):
    As = O.to_scipy(M)
    I, G, D = O.subdomain_sets(As, np.asarray(part), i, ov)
    Aii, X = O.local_matrices(As, I, G, D)
    return Aii, X, len(I)


@pytest.mark.parametrize("eps", [EPS23, 2.0 ** -30])
def test_inverse_splitting_is_inverse_of_regularised_root(eps):
    M, part, N, ov, tau = CASES["diff10_bfs"]
    for i in (0, 3, 7):
        Aii, X, nI = _local(M, part, i, ov)
        # (X^T X)^{1/2} from the symmetric eigendecomposition of the
        # Jordan-Wielandt matrix [[0, X], [X^T, 0]]: eigenpairs (sigma_j,
        # [u_j; v_j] / sqrt 2), (-sigma_j, [u_j; -v_j] / sqrt 2) and zeros, so
        # the root is the sum over positive eigenvalues of 2 theta b b^T (b the
        # lower half), without squaring X's condition number
        ni, nt = X.shape
        J = np.zeros((ni + nt, ni + nt))
        J[:ni, ni:] = X
        J[ni:, :ni] = X.T
        th, Q = np.linalg.eigh(J)
        pos = th > 0
        B = Q[ni:, pos]
        root = (B * (2.0 * th[pos])) @ B.T
        s1 = th.max()
        Abar = root + s1 * eps * np.eye(nt)
        Ginv = np.linalg.inv(Abar)
        G = MF.inverse_splitting(X, eps)
        # both sides carry rounding of order u * cond(Abar) = u / eps in norm
        assert np.linalg.norm(G - Ginv) <= 1e3 * 2.0 ** -53 / eps * np.linalg.norm(Ginv) + 1e-300


@pytest.mark.parametrize("name", list(CASES))
def test_eigenvalues_and_span_match_schur_form(name):
    M, part, N, ov, tau = CASES[name]
    nsel = 0
    for i in range(N):
        Aii, X, nI = _local(M, part, i, ov)
        lam_k, U_k, keep_k = MF.local_eigs(Aii, X, nI, tau, EPS23)
        lam_s, U_s, keep_s = O.local_eigenproblem(Aii, O.splitting_root(X, EPS23)[0], nI, tau)
        mu_k, mu_s = 1.0 / lam_k, np.where(np.isinf(lam_s), 0.0, 1.0 / lam_s)
        # mu = 1/lambda in [~eps, 1]: agreement to 1e-7 relative plus the
        # eps-cluster's own rounding (u / eps of the largest mu)
        assert np.all(np.abs(mu_k - mu_s) <= 1e-7 * mu_s + 1e-6 * EPS23), f"subdomain {i}"
        assert np.array_equal(keep_k, keep_s), f"subdomain {i}"
        p = int(keep_k.sum())
        nsel += p
        if 0 < p < nI:
            # the selected spans agree (A_II-orthogonal projectors)
            AII = Aii[:nI, :nI]
            Pk = U_k[:, :p] @ U_k[:, :p].T @ AII
            Ps = U_s[:nI, :p] @ U_s[:nI, :p].T @ AII
            gap = abs(mu_s[p] - mu_s[p - 1]) / mu_s[p]
            assert np.linalg.norm(Pk - Ps) <= 1e-6 / max(gap, 1e-3), f"subdomain {i}"
            # A_II-orthonormal columns
            assert np.allclose(U_k.T @ AII @ U_k, np.eye(nI), atol=1e-8)
    assert nsel > 0


def test_closed_form_uncoupled_blocks():
    A, part = synth.disjoint_blocks(5, 3)
    As = O.to_scipy(A)
    for i in range(3):
        I, G, D = O.subdomain_sets(As, part, i, 1)
        assert len(G) == 0 and len(D) == 0
        Aii, X = O.local_matrices(As, I, G, D)
        a = np.linalg.eigvalsh(Aii)[::-1]
        # a large shift (eps = 1/4) makes lambda spread over (0, 1) and the
        # selection lambda > 1/2 (a_j > s1 eps) partial; sigma_1 of X_i = A_ii
        # is its largest eigenvalue
        eps = 0.25
        d = a[0] * eps
        lam, U, keep = MF.local_eigs(Aii, X, len(I), 2.0, eps)
        ref = np.sort(a / (a + d))[::-1]
        assert np.allclose(lam, ref, rtol=0, atol=1e-12)
        assert np.array_equal(keep, ref > 0.5) and 0 < keep.sum() < len(I)
        # the selected u solve A_ii u = lambda (A_ii + s1 eps I) u
        for j in np.flatnonzero(keep):
            u = U[:, j]
            assert np.linalg.norm(Aii @ u - lam[j] * (Aii @ u + d * u)) <= 1e-10 * np.linalg.norm(Aii @ u)


def test_machine_eps_loses_threshold_eigenvalues():
    """eps = 2^-52 in FP64: some eigenvalue with lambda in (1/(4 tau), 100)
    moves by more than 10% relative against the Schur form, and some
    subdomain's selection count changes."""
    M, part, N, ov, tau = CASES["lap24_box6"]
    worst, changed = 0.0, 0
    for i in range(N):
        Aii, X, nI = _local(M, part, i, ov)
        lam_k, _, keep_k = MF.local_eigs(Aii, X, nI, tau, O.EPS)
        lam_s, _, keep_s = O.local_eigenproblem(Aii, O.splitting_root(X, O.EPS)[0], nI, tau)
        sel = (lam_s > 0.25 / tau) & (lam_s < 100)
        worst = max(worst, float(np.max(np.abs(lam_k[sel] - lam_s[sel]) / lam_s[sel])))
        changed += int(keep_k.sum() != keep_s.sum())
    assert worst > 0.1 and changed > 0
