"""The host-only nested-dissection order and symbolic Cholesky factorisation
(amdd_nd_order) against the graph-elimination oracle (oracle/symbolic.py),
on the CPU (no GPU involved):
  * perm is a permutation, and parent / colcount are exactly the oracle's for
    that permutation (grids, channelled 3D diffusion, stars, paths, graphs
    with several components; several leaf sizes);
  * the order reduces fill: on the 48 x 48 grid nnz(L) is below 45 % of the
    natural order's (closed form 1 + 2 (m - 1) + (n - m)(m + 1));
  * on the local matrix of an interior 64 x 64 box with one overlap layer
    (4352 unknowns, the subdomains of the 1M-unknown apply workload) the
    factor holds under 4 % of the entries of the dense triangle (under 1 %
    with leaf 16, with under 1e-3 of the dense factorisation work and an
    elimination tree under 250 levels high);
  * malformed input is rejected."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import amdd_oracle as O
from oracle import symbolic as SY


@pytest.fixture(scope="module")
def A():
    from paper_2109_05908_gb300 import amdd, build
    if not os.path.exists(amdd.LIB_PATH):
        build.build()
    return amdd


def _csr(n, edges):
    rows = [i for i, j in edges] + [j for i, j in edges] + list(range(n))
    cols = [j for i, j in edges] + [i for i, j in edges] + list(range(n))
    M = synth._csr_from_coo(n, rows, cols, np.ones(len(rows)))
    return M.rowptr, M.colind


def _graphs():
    M = synth.laplace2d(12)
    yield "grid12", M.n, M.rowptr, M.colind
    M = synth.diffusion3d(6, sigma=1.0, corr=2.0, n_channels=2, seed=1)
    yield "diff6", M.n, M.rowptr, M.colind
    n = 40
    yield "star", n, *_csr(n, [(7, k) for k in range(n) if k != 7])
    yield "path", n, *_csr(n, [(k, k + 1) for k in range(n - 1)])
    rng = np.random.default_rng(3)
    B = np.triu(rng.uniform(size=(90, 90)) < 0.03, 1)
    B[:45, 45:] = False  # two blocks: at least two components
    yield "random_split", 90, *_csr(90, list(zip(*np.nonzero(B))))
    yield "isolated", 5, np.zeros(6, np.int64), np.zeros(0, np.int32)


@pytest.mark.parametrize("leaf", [1, 4, 64])
@pytest.mark.parametrize("g", list(_graphs()), ids=lambda g: g[0])
def test_symbolic_matches_oracle(A, g, leaf):
    name, n, rp, ci = g
    perm, parent, cc, nnz = A.nd_order(n, rp, ci, leaf)
    assert np.array_equal(np.sort(perm), np.arange(n))
    p_o, cc_o = SY.eliminate(n, rp, ci, perm)
    assert np.array_equal(parent, p_o)
    assert np.array_equal(cc, cc_o)
    assert nnz == cc.sum()


def test_fill_reduction_on_a_grid(A):
    m = 48
    M = synth.laplace2d(m)
    n = M.n
    _, _, _, nnz = A.nd_order(n, M.rowptr, M.colind, 16)
    natural = 1 + 2 * (m - 1) + (n - m) * (m + 1)
    assert nnz < 0.45 * natural, (nnz, natural)


def test_local_matrix_of_the_apply_workload(A):
    m, box = 192, 64
    M = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    As = O.to_scipy(M)
    i = 4  # the interior box of the 3 x 3 layout
    I, G, D = O.subdomain_sets(As, part, i, 1)
    om = np.concatenate([I, G])
    L = sp.csr_matrix(As[om][:, om])
    L.sort_indices()
    ni = len(om)
    assert ni == 64 * 64 + 4 * 64
    _, _, _, nnz = A.nd_order(ni, L.indptr.astype(np.int64), L.indices.astype(np.int32), 64)
    dense = ni * (ni + 1) // 2
    assert nnz < 0.04 * dense, (nnz, dense)
    # leaf 16: factor entries, factorisation work sum_k colcount_k^2 and the
    # height of the elimination tree (the depth of a level-scheduled solve)
    _, parent, cc, nnz16 = A.nd_order(ni, L.indptr.astype(np.int64), L.indices.astype(np.int32), 16)
    assert nnz16 < 0.01 * dense
    assert (cc.astype(float) ** 2).sum() < 1e-3 * ni ** 3 / 3
    depth = np.zeros(ni, np.int64)
    for k in range(ni - 1, -1, -1):
        depth[k] = 0 if parent[k] < 0 else depth[parent[k]] + 1
    assert depth.max() + 1 < 250


def test_rejects_malformed(A):
    rp, ci = _csr(4, [(0, 1), (1, 2)])
    with pytest.raises(A.AmddError):
        A.nd_order(4, rp, ci, 0)
    bad = ci.copy()
    bad[0] = 9
    with pytest.raises(A.AmddError):
        A.nd_order(4, rp, bad, 8)
    rp2 = rp.copy()
    rp2[2] = rp2[1] - 1
    with pytest.raises(A.AmddError):
        A.nd_order(4, rp2, ci, 8)
    perm, parent, cc, nnz = A.nd_order(0, np.zeros(1, np.int64), np.zeros(0, np.int32), 8)
    assert nnz == 0 and len(perm) == 0
