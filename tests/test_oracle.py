"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a hand-derived fixture, an independent brute-force computation in
extended precision, an inequality proved in the paper, or a special case that
reduces to a textbook result.  The last group plants plausible mistakes in the
oracle (on the CPU) and checks that the pins catch them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import synth
from oracle import amdd_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_2d(m=12, box=4):
    A = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    return A, part, int(part.max()) + 1


def _small_3d(seed=1):
    A = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=seed, channel_value=1e3)
    part = synth.bfs_partition(A, 6, seed=seed, min_size=40, max_size=160)
    return A, part, int(part.max()) + 1


# ---------------------------------------------------------------- Sec. 2.1 sets
def test_sets_match_hand_derived_fixture():
    """Sec. 2.1: Omega_Ii, Omega_Gi, Omega_Di on a 4x4 grid, hand-derived."""
    A = O.to_scipy(synth.laplace2d(4))
    part = synth.box_partition_2d(4, 2)
    want = {}
    with open(os.path.join(GOLDEN, "sets_4x4_box2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            want[(int(tok[0]), tok[1])] = [int(t) for t in tok[2:]]
    for ov in (1, 2):
        I, G, D = O.subdomain_sets(A, part, 0, ov)
        assert list(I) == want[(ov, "I")]
        assert list(G) == want[(ov, "G")]
        assert list(D) == want[(ov, "D")]


@pytest.mark.parametrize("ov", [1, 2, 3])
def test_sets_match_graph_distances(ov):
    """Layers equal graph distances computed by an independent shortest-path
    routine (unweighted BFS in scipy.sparse.csgraph)."""
    A, part, N = _small_3d()
    As = O.to_scipy(A)
    adj = sp.csr_matrix((np.ones(As.nnz), As.indices, As.indptr), shape=As.shape)
    for i in range(N):
        I, G, D = O.subdomain_sets(As, part, i, ov)
        d = shortest_path(adj, unweighted=True, indices=np.flatnonzero(part == i)).min(axis=0)
        assert np.array_equal(I, np.flatnonzero(d == 0))
        assert np.array_equal(G, np.flatnonzero((d >= 1) & (d <= ov)))
        assert np.array_equal(D, np.flatnonzero(d == ov + 1))


# ------------------------------------------------------- spectra and closed forms
def test_single_subdomain_singular_values_closed_form():
    """N = 1: Omega_G = Omega_D = {} so X = A, and the singular values of the
    SPD 5-point Laplacian are its eigenvalues 4 - 2cos(j pi/(m+1)) - 2cos(k pi/(m+1))."""
    m = 9
    A = O.to_scipy(synth.laplace2d(m))
    part = np.zeros(m * m, dtype=np.int32)
    I, G, D = O.subdomain_sets(A, part, 0, 1)
    assert len(G) == 0 and len(D) == 0
    _, X = O.local_matrices(A, I, G, D)
    _, s = O.splitting_root(X)
    j = np.arange(1, m + 1)
    lam = (4 - 2 * np.cos(j[:, None] * np.pi / (m + 1)) - 2 * np.cos(j[None, :] * np.pi / (m + 1))).ravel()
    assert np.allclose(np.sort(s), np.sort(lam), rtol=0, atol=1e-13)


def test_local_matrix_rows_are_rows_of_A():
    """Eq. (Xi): each row of X_i holds the whole row of A (no entry dropped),
    because the columns span Omega_i plus one more layer."""
    A, part, N = _small_3d()
    As = O.to_scipy(A)
    for i in range(N):
        I, G, D = O.subdomain_sets(As, part, i, 1)
        Aii, X = O.local_matrices(As, I, G, D)
        om = np.concatenate([I, G])
        assert np.allclose(np.abs(X).sum(1), np.asarray(abs(As[om]).sum(1)).ravel(), rtol=1e-14)
        assert np.array_equal(Aii, X[:, : len(om)])


# ------------------------------------------------------------ Lemmas 3.1 and 3.2
@pytest.mark.parametrize("maker", [_small_2d, _small_3d])
def test_splitting_lemmas(maker):
    """Lemma 3.1: Abar_ii is the square root of X_i^T X_i (up to the shift of
    Remark 3.2) and tilde R_i^T Abar_ii tilde R_i <= A.  Lemma 3.2: the Schur
    complement tilde A_ii is SPSD and R_i^T tilde A_ii R_i <= A."""
    A, part, N = maker()
    As = O.to_scipy(A)
    Ad = As.toarray()
    for i in range(N):
        I, G, D = O.subdomain_sets(As, part, i, 1)
        Aii, X = O.local_matrices(As, I, G, D)
        Abar, s = O.splitting_root(X)
        sh = s[0] * O.EPS
        B = Abar - sh * np.eye(len(Abar))
        assert np.allclose(B @ B, X.T @ X, atol=1e-12 * s[0] ** 2)
        omt = np.concatenate([I, G, D])
        om = np.concatenate([I, G])
        P = np.zeros_like(Ad)
        P[np.ix_(omt, omt)] = Abar
        tol = 1e-11 * s[0]
        assert np.linalg.eigvalsh(Ad - P).min() >= -tol
        tA = O.schur_overlap(Abar, len(om))
        assert np.linalg.eigvalsh(tA).min() >= -tol
        Q = np.zeros_like(Ad)
        Q[np.ix_(om, om)] = tA
        assert np.linalg.eigvalsh(Ad - Q).min() >= -tol


def test_all_nonzero_eigenvalues_at_least_one():
    """With Boolean D_i, every non-zero eigenvalue of eq. (Zi) is >= 1: on
    vectors supported on Omega_Ii, D_i A_ii D_i = A and the splitting gives
    u^T tilde A_ii u <= u^T A u, so by Courant-Fischer the nI non-zero
    eigenvalues are >= 1 (up to the eps shift)."""
    for maker in (_small_2d, _small_3d):
        A, part, N = maker()
        S = O.setup(A, part, N, 1, tau=50.0)
        for s in S.subs:
            assert s.lam.min() >= 1.0 - 1e-9
            assert len(s.lam) == len(s.I)


def test_schur_quotient_property():
    """Eliminating Omega_Gi from eq. (tildeA)'s tilde A_ii gives the same pencil
    as eliminating Omega_Gi and Omega_Di from Abar_ii at once (quotient
    property); checked on eigenvalues of eq. (Zi) below the eps-cluster."""
    A, part, N = _small_2d()
    As = O.to_scipy(A)
    for i in range(N):
        I, G, D = O.subdomain_sets(As, part, i, 1)
        Aii, X = O.local_matrices(As, I, G, D)
        Abar, sg = O.splitting_root(X)
        tA = O.schur_overlap(Abar, len(I) + len(G))
        nI = len(I)
        S1 = tA[:nI, :nI] - tA[:nI, nI:] @ np.linalg.solve(tA[nI:, nI:], tA[nI:, :nI])
        mu1 = sla.eigh(0.5 * (S1 + S1.T), Aii[:nI, :nI], eigvals_only=True)
        lam, _, _ = O.local_eigenproblem(Aii, Abar, nI, 1.0)
        lam1 = np.sort(1.0 / mu1[mu1 > 1e-8])
        assert np.allclose(np.sort(lam[lam < 1e8]), lam1, rtol=1e-10)


# --------------------------------------- eq. (Zi) by brute force in extended precision
def _bruteforce_zi(X, Aii, nI, dps=40):
    """Eq. (invAii) and eq. (Zi) exactly as printed, in mpmath at `dps`
    digits: full SVD of X_i, Abar^{-1} = V (S + s1 eps)^{-1} V^T +
    (s1 eps)^{-1} V_perp V_perp^T, tilde A_ii^{-1} = the Omega_i block of
    Abar^{-1} (inverse of a Schur complement), then the eigenvalues of
    tilde A_ii^{-1} D A_ii D.  Returns (lam_nonzero, eigvecs restricted to
    Omega_Ii) as float arrays."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    n_i, nt = X.shape
    Xm = mp.matrix(X.tolist())
    U, S, Vt = mp.svd_r(Xm, full_matrices=True)
    eps = mp.mpf(2) ** -52
    s1 = S[0]
    inv = mp.zeros(nt, nt)
    for k in range(nt):
        sk = S[k] if k < n_i else mp.mpf(0)
        w = 1 / (sk + s1 * eps)
        for a in range(nt):
            va = Vt[k, a] * w
            for b in range(nt):
                inv[a, b] += va * Vt[k, b]
    G = inv[0:n_i, 0:n_i]
    DAD = mp.zeros(n_i, n_i)
    for a in range(nI):
        for b in range(nI):
            DAD[a, b] = Aii[a, b]
    ev, vr = mp.eig(G * DAD)
    lam, vecs = [], []
    for k in range(n_i):
        if abs(ev[k]) > mp.mpf(10) ** -20:
            lam.append(float(mp.re(ev[k])))
            vecs.append([float(mp.re(vr[a, k])) for a in range(nI)])
    return np.array(lam), np.array(vecs).T


def test_eigenproblem_matches_extended_precision_bruteforce():
    """The oracle's eq. (Zi) eigenvalues and selected spans match a 40-digit
    evaluation of the paper's formulas on a tiny problem: finite eigenvalues
    to 1e-10 relative, the count of the eps-cluster exactly, spans to 1e-8."""
    m = 6
    A = O.to_scipy(synth.laplace2d(m))
    part = synth.box_partition_2d(m, 3)
    for i in (0, 1):
        I, G, D = O.subdomain_sets(A, part, i, 1)
        Aii, X = O.local_matrices(A, I, G, D)
        Abar, sg = O.splitting_root(X)
        for tau in (0.5, 50.0):
            lam, U, keep = O.local_eigenproblem(Aii, Abar, len(I), tau)
            blam, bvec = _bruteforce_zi(X, Aii, len(I))
            assert len(blam) == len(lam) == len(I)
            order = np.argsort(-blam)
            blam, bvec = blam[order], bvec[:, order]
            fin = blam < 1e8
            assert np.allclose(np.sort(lam[lam < 1e8]), np.sort(blam[fin]), rtol=1e-10, atol=0)
            # eps-cluster: magnitude ~ 1/(s1 eps) fixed by the shift of Sec. 3.2;
            # FP64 resolves it only to ~10%, so compare within a factor 1.5
            ocl, bcl = np.sort(lam[lam >= 1e8]), np.sort(blam[~fin])
            assert len(ocl) == len(bcl)
            assert np.all(np.abs(np.log(ocl / bcl)) < np.log(1.5))
            bkeep = blam > 1.0 / tau
            assert bkeep.sum() == keep.sum()
            if 0 < keep.sum() < len(I):
                q1, _ = np.linalg.qr(U[: len(I), keep])
                q2, _ = np.linalg.qr(bvec[:, bkeep])
                # sine of the largest principal angle between the two spans
                assert np.linalg.norm(q2 - q1 @ (q1.T @ q2), 2) < 1e-8


# ------------------------------------------------------------ preconditioner
def _dense_minv(S):
    n = S.A.shape[0]
    return np.column_stack([O.apply(S, e) for e in np.eye(n)])


def test_single_subdomain_is_twice_exact_inverse():
    """N = 1: Omega_i is everything, tilde A = A + s1 eps I, every eigenvalue of
    eq. (Zi) is ~1 > 1/tau, so the coarse space is R^n, the coarse term is
    A^{-1} and M^{-1} = 2 A^{-1}; PCG converges in one iteration."""
    m = 8
    A = synth.laplace2d(m)
    part = np.zeros(m * m, dtype=np.int32)
    S = O.setup(A, part, 1, 1, tau=50.0)
    assert S.nC == m * m
    Ad = S.A.toarray()
    assert np.allclose(_dense_minv(S), 2 * np.linalg.inv(Ad), rtol=0, atol=1e-10)
    b = synth.rhs(m * m, 3)
    x, its, _ = O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-10)
    assert its == 1
    assert np.allclose(x, np.linalg.solve(Ad, b), atol=1e-10)


@pytest.mark.parametrize("maker,tau", [(_small_2d, 0.5), (_small_2d, 50.0), (_small_3d, 0.5),
                                       (_small_3d, 0.05), (_small_3d, 100.0)])
def test_condition_bound(maker, tau):
    """Sec. 3.2: kappa(M^{-1} A) <= (k_c + 1)(2 + (2 k_c + 1) k_m / tau), with
    lambda_max <= k_c + 1 and lambda_min >= 1 / (2 + (2 k_c + 1) k_m / tau)."""
    A, part, N = maker()
    S = O.setup(A, part, N, 1, tau)
    Ad = S.A.toarray()
    Minv = _dense_minv(S)
    ev = np.sort(np.linalg.eigvals(Minv @ Ad).real)
    kc, km = O.colouring_number(S), O.splitting_constant(S)
    assert km <= N + 1e-8
    assert ev[-1] <= kc + 1 + 1e-8
    assert ev[0] >= 1.0 / (2 + (2 * kc + 1) * km / tau) - 1e-10
    assert ev[-1] / ev[0] <= O.condition_bound(kc, km, tau) * (1 + 1e-10)


@pytest.mark.parametrize("maker,tau", [(_small_2d, 0.5), (_small_3d, 0.5), (_small_3d, 100.0)])
def test_lanczos_estimate_against_dense_spectrum(maker, tau):
    """The CG-Lanczos tridiagonal (Saad, Sec. 6.7.3) built from the PCG
    coefficients has Ritz values inside the dense spectrum of M^{-1} A, and
    run to a tight tolerance its extremes reach the extreme eigenvalues."""
    A, part, N = maker()
    S = O.setup(A, part, N, 1, tau)
    ev = np.sort(np.linalg.eigvals(_dense_minv(S) @ S.A.toarray()).real)
    b = synth.rhs(A.n, 3)
    co = []
    O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-8, coeffs=co)
    lo, hi = O.lanczos_extremes(co)
    assert ev[0] * (1 - 1e-9) <= lo and hi <= ev[-1] * (1 + 1e-9)
    assert hi / lo <= ev[-1] / ev[0] * (1 + 1e-9)
    co = []
    O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-13, coeffs=co)
    lo, hi = O.lanczos_extremes(co)
    assert abs(hi - ev[-1]) <= 1e-6 * ev[-1]
    assert abs(lo - ev[0]) <= 2e-3 * ev[0]


def test_lanczos_estimate_first_step():
    """Closed forms on a diagonal system with M = I: after one step T =
    [1/alpha_1] = (b, A b)/(b, b), the mean of the diagonal for b = 1; after
    n steps on n distinct eigenvalues T is similar to A, so its extremes are
    those of A."""
    d = np.array([1.0, 2.0, 5.0])
    As = sp.diags(d).tocsr()
    b = np.array([1.0, 1.0, 1.0])
    co = []
    O.pcg(As, b, lambda r: r.copy(), rtol=1e-30, maxit=1, coeffs=co)
    lo, hi = O.lanczos_extremes(co)
    # z = b, alpha = (b,b)/(b,Ab) -> Ritz value (b,Ab)/(b,b) = mean(d)
    assert lo == pytest.approx(d.mean(), rel=1e-14) and hi == lo
    co = []
    O.pcg(As, b, lambda r: r.copy(), rtol=1e-30, maxit=3, coeffs=co)
    lo, hi = O.lanczos_extremes(co)
    # three steps on a 3x3 system with distinct eigenvalues: T is similar to diag(d)
    assert lo == pytest.approx(1.0, rel=1e-12) and hi == pytest.approx(5.0, rel=1e-12)


def test_preconditioner_symmetric_positive_definite():
    """M^{-1} of eq. (two_level_schwarz) is symmetric positive definite."""
    A, part, N = _small_3d()
    S = O.setup(A, part, N, 1, 0.5)
    Minv = _dense_minv(S)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max()
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0


def test_coarse_operator_basis_invariant():
    """R_0^T (R_0 A R_0^T)^{-1} R_0 depends only on the span of each Z_i."""
    A, part, N = _small_2d()
    S = O.setup(A, part, N, 1, 0.5)
    rng = np.random.default_rng(0)
    C1 = (S.W @ sla.cho_solve(S.E_chol, S.W.T.toarray())).copy()
    for s in S.subs:
        T = rng.standard_normal((s.p, s.p)) + 3 * np.eye(s.p)
        s.Z = s.Z @ T
    W = O.coarse_basis(S.subs, S.A.shape[0])
    E = (W.T @ (S.A @ W)).toarray()
    C2 = W @ np.linalg.solve(E, W.T.toarray())
    assert np.allclose(C1, C2, atol=1e-10 * np.abs(C1).max())


def test_pcg_solution_and_cg_bound():
    """PCG reaches 1e-8 and agrees with a dense solve; the iteration count
    respects the CG bound of Sec. 1 with kappa from the dense spectrum."""
    A, part, N = _small_3d()
    S = O.setup(A, part, N, 1, 0.5)
    b = synth.rhs(A.n, 5)
    x, its, hist = O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-8)
    Ad = S.A.toarray()
    xs = np.linalg.solve(Ad, b)
    assert hist[-1] <= 1e-8
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    ev = np.sort(np.linalg.eigvals(_dense_minv(S) @ Ad).real)
    kappa = ev[-1] / ev[0]
    rho = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    # ||e_k||_A <= 2 rho^k ||e_0||_A, and ||r||_2 / ||b||_2 <= sqrt(cond(A)) ||e||_A/||e_0||_A
    condA = np.linalg.cond(Ad)
    kmax = int(np.ceil(np.log(1e-8 / (2 * np.sqrt(condA))) / np.log(rho)))
    assert its <= kmax


def test_one_level_needs_more_iterations():
    """Negative control (Sec. 4.1): without the coarse term, PCG takes more
    iterations on the same problem."""
    A, part, N = _small_2d(32, 4)
    S = O.setup(A, part, N, 1, 0.5)
    b = synth.rhs(A.n, 1)
    _, its2, _ = O.pcg(S.A, b, lambda r: O.apply(S, r))
    _, its1, _ = O.pcg(S.A, b, lambda r: O.apply_one_level(S, r))
    assert its1 > its2 + 10


# ------------------------------------------------------------ planted mistakes
def test_planted_schur_sign_is_caught(monkeypatch):
    """A '+' instead of '-' in eq. (tildeA) breaks Lemma 3.2's inequality."""
    def wrong(Abar, n_i):
        X11, X12, X21, X22 = Abar[:n_i, :n_i], Abar[:n_i, n_i:], Abar[n_i:, :n_i], Abar[n_i:, n_i:]
        return X11 + X12 @ np.linalg.solve(X22, X21)
    monkeypatch.setattr(O, "schur_overlap", wrong)
    with pytest.raises(AssertionError):
        test_splitting_lemmas(_small_2d)


def test_planted_missing_square_root_is_caught(monkeypatch):
    """Using V S^2 V^T (X^T X itself) instead of its square root breaks Lemma 3.1."""
    def wrong(X, eps=O.EPS):
        _, s, Vt = np.linalg.svd(X, full_matrices=True)
        V = Vt[: X.shape[0]].T
        return (V * s ** 2) @ V.T + s[0] * eps * np.eye(X.shape[1]), s
    monkeypatch.setattr(O, "splitting_root", wrong)
    with pytest.raises(AssertionError):
        test_splitting_lemmas(_small_2d)


def test_planted_reversed_selection_is_caught(monkeypatch):
    """Keeping lambda < 1/tau instead of lambda > 1/tau changes the selected
    count against the extended-precision evaluation of eq. (Zi)."""
    orig = O.local_eigenproblem

    def wrong(Aii, Abar, nI, tau):
        lam, U, keep = orig(Aii, Abar, nI, tau)
        return lam, U, ~keep
    monkeypatch.setattr(O, "local_eigenproblem", wrong)
    with pytest.raises(AssertionError):
        test_eigenproblem_matches_extended_precision_bruteforce()


def test_planted_dropped_shift_is_caught(monkeypatch):
    """Dropping the complement term s1 eps V_perp V_perp^T of Sec. 3.2 leaves
    Abar_ii singular on Omega_Di, so the Schur complement of eq. (tildeA)
    cannot be formed (Cholesky of X22 fails) or departs from the 40-digit
    evaluation."""
    def wrong(X, eps=O.EPS):
        _, s, Vt = np.linalg.svd(X, full_matrices=True)
        V = Vt[: X.shape[0]].T
        return (V * (s + s[0] * eps)) @ V.T, s
    monkeypatch.setattr(O, "splitting_root", wrong)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        test_eigenproblem_matches_extended_precision_bruteforce()


# ------------------------------------------------- k_c and k_m of Sec. 3.2
@pytest.mark.parametrize("m,box,kc", [(8, 4, 4), (16, 4, 4), (12, 12, 1)])
def test_colouring_number_of_box_layouts(m, box, kc):
    """k_c on box layouts with overlap 1 where it is known: on a 2 x 2 grid of
    boxes every overlapped subdomain touches the three others (K_4, four
    colours); on a 4 x 4 grid each box touches its eight king-move neighbours
    and no box two steps away (the king's graph, chromatic number 4, which
    the row-major greedy order attains); one box needs one colour.  A
    colouring that missed the diagonal neighbours would find 2 here."""
    A = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    S = O.setup(A, part, int(part.max()) + 1, 1, 0.5)
    assert O.colouring_number(S) == kc


def test_colouring_number_of_strips():
    """Vertical strips four columns wide with overlap 1: strip i touches only
    strips i - 1 and i + 1, a path, so two colours."""
    m = 16
    A = synth.laplace2d(m)
    part = (np.arange(m * m) % m // 4).astype(np.int32)
    S = O.setup(A, part, 4, 1, 0.5)
    assert O.colouring_number(S) == 2


@pytest.mark.parametrize("m,eps", [(8, 1e-3), (10, 2.0 ** -20)])
def test_splitting_constant_single_subdomain(m, eps):
    """N = 1: Omega_G and Omega_D are empty, X = A, the regularised root is
    (A^T A)^{1/2} + sigma_1 eps I = A + sigma_1 eps I with sigma_1 = lambda_max(A),
    so k_m = lambda_max(A + sigma_1 eps I, A) = 1 + eps lambda_max / lambda_min,
    in closed form from the Laplacian's spectrum 4 - 2cos(j pi/(m+1)) -
    2cos(k pi/(m+1)).  A dropped shift would give exactly 1."""
    A = synth.laplace2d(m)
    part = np.zeros(m * m, np.int32)
    S = O.setup(A, part, 1, 1, 0.5, eps=eps)
    c = np.cos(np.pi / (m + 1))
    lmin, lmax = 4.0 - 4.0 * c, 4.0 + 4.0 * c
    km = O.splitting_constant(S)
    assert km - 1.0 == pytest.approx(eps * lmax / lmin, rel=1e-6)


def test_splitting_constant_at_most_multiplicity():
    """Each R_i^T tilde A_ii R_i is at most A in the Loewner order (Lemma 3.2),
    so k_m is at most the number of subdomains whose Omega_i holds a given
    unknown, maximised over unknowns (here: overlap-1 boxes on a 12 x 12 grid,
    multiplicity 4 at box corners).  The lower check (k_m >= 1) is a sanity
    bar on this layout, where vectors supported deep inside one box see only
    that box's term."""
    A, part, N = _small_2d()
    S = O.setup(A, part, N, 1, 0.5)
    mult = np.zeros(A.n, int)
    for s in S.subs:
        mult[s.omega] += 1
    km = O.splitting_constant(S)
    assert 1.0 <= km <= mult.max() + 1e-10
