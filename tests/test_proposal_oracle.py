"""Pins of the learned warm-start oracle (oracle/proposal.py) against closed
forms, finite differences, a library rounding routine and a dense
eigensolver (CPU)."""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import proposal as L


def test_bf16_rounding_definition():
    """Round to nearest, ties to even, on the 7 stored mantissa bits."""
    one = 1.0
    assert L.bf16(one)[()] == 1.0
    assert L.bf16(1 + 2.0 ** -8)[()] == 1.0              # tie -> even (1.0)
    assert L.bf16(1 + 3 * 2.0 ** -8)[()] == 1 + 2.0 ** -6  # tie -> even (odd neighbour below)
    assert L.bf16(1 + 2.0 ** -8 + 2.0 ** -12)[()] == 1 + 2.0 ** -7
    assert L.bf16(-2.5)[()] == -2.5
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 100
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(x), ref)


def test_mlp_gradients_match_finite_differences():
    """backward() against central differences of loss(forward()) in FP64."""
    rng = np.random.default_rng(1)
    P = L.init_params(3)
    for k in P:
        P[k] = P[k] * 0.5 + (0.01 * rng.standard_normal(P[k].shape) if k.startswith("b") else 0.0)
    X = rng.standard_normal((5, L.NF))
    Qt = rng.standard_normal((5, L.NB, L.NB))
    Qt = 0.5 * (Qt + Qt.transpose(0, 2, 1))
    Qh, cache = L.forward(P, X)
    g = L.backward(P, Qh, Qt, cache)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, 6, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = L.loss(L.forward(P, X)[0], Qt)
            flat[idx] = old - h
            lm = L.loss(L.forward(P, X)[0], Qt)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_adam_first_step_closed_form():
    """After one step from zero moments the bias-corrected ratio is
    g / (|g| + eps): each parameter moves by lr * sign(g)."""
    P = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 0.0])}
    st = {}
    L.adam_step(P, g, st, lr=0.1)
    assert np.allclose(P["w"], [1.0 - 0.1, -2.0 + 0.1, 3.0], atol=1e-6)


def test_krylov_basis_spans_krylov_space():
    A, part, N = synth.laplace2d(8), synth.box_partition_2d(8, 4), 4
    Aii = O.to_scipy(A).toarray()[:20, :20]
    B = L.krylov_basis(Aii, 5)
    assert np.allclose(B.T @ B, np.eye(5), atol=1e-12)
    K = np.column_stack([np.linalg.matrix_power(Aii, j) @ np.ones(20) for j in range(5)])
    Qk, _ = np.linalg.qr(K)
    assert np.allclose(B @ B.T, Qk @ Qk.T, atol=1e-10)
    # an invariant starting vector ends the space after one vector
    B2 = L.krylov_basis(np.eye(7) * 3.0, 4)
    assert np.allclose(B2[:, 0], 1 / np.sqrt(7)) and np.all(B2[:, 1:] == 0)


def test_target_projector_closed_form_and_invariance():
    rng = np.random.default_rng(2)
    B, _ = np.linalg.qr(rng.standard_normal((40, L.NB)))
    U = B[:, :3]
    Q = L.target_projector(B, U)
    assert np.allclose(Q, np.diag([1, 1, 1] + [0] * (L.NB - 3)), atol=1e-12)
    R = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    assert np.allclose(L.target_projector(B, U @ R), Q, atol=1e-12)
    # the proposal from the exact projector recovers span(U)
    Xp = L.proposal(Q, B, 3)
    Pq = Xp @ np.linalg.pinv(Xp)
    assert np.allclose(Pq, U @ U.T, atol=1e-10)


def test_features_invariant_to_local_order_and_closed_form():
    A = synth.laplace2d(12)
    part = synth.box_partition_2d(12, 4)
    As = O.to_scipy(A)
    I, G, D = O.subdomain_sets(As, part, 4, 1)
    Aii, _ = O.local_matrices(As, I, G, D)
    f = L.features(Aii, len(I), len(G), len(D), 10, 0.5)
    assert f.shape == (32,)
    assert np.isclose(f[5], np.log(4.0)) and f[6] == 0.0   # every diagonal entry is 4
    assert f[26] == 0.0                                     # no positive off-diagonal
    assert np.isclose(f[0], np.log(16)) and f[31] == 1.0
    perm = np.random.default_rng(0).permutation(len(I))
    gp = np.random.default_rng(1).permutation(len(G))
    order = np.concatenate([perm, len(I) + gp])
    f2 = L.features(Aii[np.ix_(order, order)], len(I), len(G), len(D), 10, 0.5)
    assert np.allclose(f, f2, rtol=1e-12, atol=1e-12)


def test_lobpcg_closed_form_spectrum():
    """Diagonal T: the p smallest eigenvalues are the p smallest entries."""
    rng = np.random.default_rng(3)
    d = np.linspace(0.0, 1.0, 60) ** 2
    T = np.diag(rng.permutation(d))
    X0 = rng.standard_normal((60, 8))
    th, X, its, ok = L.lobpcg(T, X0, 6, tol=1e-9)
    assert ok
    assert np.allclose(th, np.sort(d)[:6], atol=1e-12)
    assert np.linalg.norm(T @ X - X * th, axis=0).max() <= 1e-9


def test_lobpcg_matches_dense_on_local_pencil():
    """On a subdomain's T of eq. (Zi) the p smallest Ritz values match the
    dense eigenvalues, and an exact start converges at once."""
    A = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=1, channel_value=1e3)
    part = synth.bfs_partition(A, 6, seed=1, min_size=40, max_size=160)
    S = O.setup(A, part, int(part.max()) + 1, 1, 0.5)
    s = next(t for t in S.subs if 0 < t.p < len(t.I))
    nI = len(s.I)
    Abar, _ = O.splitting_root(O.local_matrices(S.A, s.I, s.G, s.D)[1])
    T, LA = L.reduced_T(s.Aii, Abar, nI)
    W = LA.T @ s.Z[:nI]  # T w = mu w with w = L_A^T u
    mu_sel = np.sort(np.where(np.isinf(s.lam), 0.0, 1.0 / s.lam))[: s.p]
    ev = np.linalg.eigvalsh(T)
    # the eps-cluster (mu ~ sigma_1 eps) is fixed by FP64 only to ~1e-6 between
    # two formulations of the same pencil; the finite part to 1e-8
    fin = mu_sel > 1e-4
    assert np.allclose(ev[: s.p][fin], mu_sel[fin], rtol=1e-8, atol=1e-10)
    assert np.allclose(ev[: s.p][~fin], mu_sel[~fin], atol=2e-6)
    assert ev[s.p] > 0.5 > ev[s.p - 1]  # tau = 0.5 splits the spectrum at p
    rng = np.random.default_rng(4)
    k = s.p + 4
    th, X, its, ok = L.lobpcg(T, rng.standard_normal((nI, k)), s.p, tol=1e-7, maxit=500)
    assert ok and np.allclose(th, ev[: s.p], atol=1e-9)
    # the block spans ~all of R^nI here (3k > nI): the Ritz vectors must stay orthonormal
    assert np.allclose(X.T @ X, np.eye(s.p), atol=1e-10)
    Wq, _ = np.linalg.qr(W)
    Xq, _ = np.linalg.qr(X)
    assert np.linalg.norm(Wq - Xq @ (Xq.T @ Wq), 2) <= 1e-5
    th2, _, its2, ok2 = L.lobpcg(T, np.hstack([W, rng.standard_normal((nI, 4))]), s.p, tol=1e-7)
    assert ok2 and its2 <= 2 and its < 500
