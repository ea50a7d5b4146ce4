"""Pins of the oracle's multilevel form (Sec. 3.2, last paragraph; Sec. 4.2):
the block-pattern coarse matrix, the grouped second-level partition, the
reduction to the two-level method with an exact inner solve, the invariance
under orthogonal changes of the coarse basis, and the outer iteration count
of the three-level solver (CPU)."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import amdd_oracle as O
from oracle import multilevel as ML


def _lap(m=24, box=6, tau=0.5, g=2, ov=1):
    A = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    nb = m // box
    groups = synth.box_groups_2d(nb, g)
    return A, part, nb * nb, ov, tau, groups, int(groups.max()) + 1


@pytest.fixture(scope="module")
def three_level():
    A, part, N, ov, tau, groups, N2 = _lap()
    return ML.setup(A, part, N, ov, tau, groups, N2, 1, 0.5), part, groups


def test_block_pattern_holds_all_of_E(three_level):
    """Blocks of subdomains not coupled in A are exactly zero in E, so the
    block pattern loses nothing; the pattern has exactly the coupled blocks."""
    M, part, groups = three_level
    S = M.S1
    assert np.array_equal(M.E.toarray(), S.E)
    off = np.concatenate([[0], np.cumsum([s.p for s in S.subs])])
    pairs = ML.coupled_pairs(S.A, part)
    N = len(S.subs)
    nnz = sum(S.subs[i].p * S.subs[j].p for i in range(N) for j in range(N) if i == j or (i, j) in pairs)
    assert M.E.nnz == nnz
    for i in range(N):
        for j in range(N):
            if i != j and (i, j) not in pairs:
                assert not np.any(S.E[off[i]:off[i + 1], off[j]:off[j + 1]])


@pytest.mark.parametrize("ov", [1, 2])
def test_block_pattern_overlap2_and_3d(ov):
    A = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=1, channel_value=1e3)
    part = synth.bfs_partition(A, 6, seed=1, min_size=40, max_size=160)
    N = int(part.max()) + 1
    S = O.setup(A, part, N, ov, 0.5)
    E = ML.coarse_matrix_blocks(S, part)
    assert np.array_equal(E.toarray(), S.E)
    assert (E - E.T).nnz == 0 or np.abs((E - E.T).data).max() == 0.0


def test_grouped_partition(three_level):
    M, part, groups = three_level
    p2 = ML.coarse_partition(M.S1, groups)
    assert len(p2) == M.S1.nC
    for g in range(int(groups.max()) + 1):
        assert np.sum(p2 == g) == sum(s.p for i, s in enumerate(M.S1.subs) if groups[i] == g)
    # the groups of the box helper: 2 x 2 boxes of a 4 x 4 box partition
    assert synth.box_groups_2d(4, 2).tolist() == [0, 0, 1, 1, 0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 3, 3]


def test_exact_inner_solve_is_the_two_level_method(three_level):
    """With a tight inner tolerance the coarse solve is exact and the
    multilevel apply equals the two-level deflated apply."""
    M, part, groups = three_level
    M.inner_rtol, M.inner_maxit = 1e-14, 400
    try:
        r = np.random.default_rng(3).uniform(-1, 1, M.S1.A.shape[0])
        z2 = O.apply_deflated(M.S1, r)
        zm = ML.apply_deflated(M, r)
        assert np.linalg.norm(zm - z2) <= 1e-10 * np.linalg.norm(z2)
        # the inner solve itself against a dense solve
        c = M.S1.W.T @ r
        e = ML.coarse_solve(M, c)
        assert np.linalg.norm(e - np.linalg.solve(M.S1.E, c)) <= 1e-11 * np.linalg.norm(e)
    finally:
        M.inner_rtol, M.inner_maxit = 1e-4, 100


def test_single_second_level_subdomain_is_exact():
    """N2 = 1: the second-level restricted method is E^{-1} itself, so the
    inner GMRES needs one iteration."""
    A, part, N, ov, tau, _, _ = _lap(m=16, box=4)
    M = ML.setup(A, part, N, ov, tau, np.zeros(N, np.int32), 1, 1, 0.5, inner_rtol=1e-10)
    c = np.random.default_rng(5).uniform(-1, 1, M.S1.nC)
    e = ML.coarse_solve(M, c)
    assert M.inner_its[-1] == 1
    assert np.linalg.norm(M.E @ e - c) <= 1e-10 * np.linalg.norm(c)


def test_orthogonal_coarse_basis_invariance(three_level):
    """Replacing each first-level Z_i by Z_i Q_i (Q_i orthogonal) transforms
    E by a block-orthogonal congruence; the second-level construction
    (square root of X^T X, Schur complements, eq. (Zi), deflation) commutes
    with it: M2' (Q^T v) = Q^T M2 v.  A library whose coarse basis differs
    from the oracle's by such Q_i (any two A_II-orthonormal bases of the same
    span do) builds the same multilevel preconditioner."""
    M, part, groups = three_level
    S = M.S1
    rng = np.random.default_rng(11)
    Qs = [sla.qr(rng.standard_normal((s.p, s.p)))[0] if s.p else np.zeros((0, 0)) for s in S.subs]
    Q = sla.block_diag(*[q for q in Qs if q.size])
    Ep = Q.T @ S.E @ Q
    import scipy.sparse as sp
    C = M.E.tocoo()                            # stored pattern, explicit zeros included
    Eps = sp.coo_matrix((Ep[C.row, C.col], (C.row, C.col)), shape=C.shape).tocsr()
    p2 = ML.coarse_partition(S, groups)
    S2p = O.setup(Eps, p2, int(groups.max()) + 1, 1, 0.5)
    v = rng.uniform(-1, 1, S.nC)
    z = O.apply_deflated(M.S2, v)
    zp = O.apply_deflated(S2p, Q.T @ v)
    assert np.linalg.norm(zp - Q.T @ z) <= 1e-9 * np.linalg.norm(z)
    assert [s.p for s in S2p.subs] == [s.p for s in M.S2.subs]


def test_three_level_outer_iterations(three_level):
    """Sec. 4.2: with inner GMRES(30) to 1e-4 on the second level, the outer
    flexible GMRES(30) reaches 1e-8 in the two-level method's iteration
    count (here within one), with a small number of inner iterations."""
    M, part, groups = three_level
    b = synth.rhs(M.S1.A.shape[0], 0)
    _, its2, _ = O.gmres(M.S1.A, b, lambda v: O.apply_deflated(M.S1, v), restart=30, rtol=1e-8)
    M.inner_its.clear()
    x, its3, hist = ML.solve(M, b)
    assert hist[-1] <= 1e-8
    assert np.linalg.norm(b - M.S1.A @ x) <= 1.5e-8 * np.linalg.norm(b)
    assert its3 <= its2 + 1, (its3, its2)
    assert 0 < max(M.inner_its) <= 30
