"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/amdd.h declares, and its host-only entry points behave.
No compute call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "amdd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amdd_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def A():
    from paper_2109_05908_gb300 import amdd, build
    if not os.path.exists(amdd.LIB_PATH):
        build.build()
    return amdd


def test_exports_every_declared_symbol(A):
    L = ctypes.CDLL(A.LIB_PATH)
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(A.SIGNATURES)


def test_noalloc_bound_matches_header(A):
    """The binding's copy of AMDD_NOALLOC_MAX_N is the header's."""
    txt = open(os.path.join(ROOT, "include", "amdd.h")).read()
    m = re.search(r"#define\s+AMDD_NOALLOC_MAX_N\s+(\d+)", txt)
    assert m and int(m.group(1)) == A.NOALLOC_MAX_N


def test_status_strings_and_defaults(A):
    for k in range(8):
        assert A.status_str(k)
    o = A.opts_default()
    assert o.eps == 2.0 ** -52 and o.max_sweeps == 60
    assert o.tie_band == 1e-10 and o.use_graphs == 1 and o.autotune == 1 and o.mem_budget == 0
    assert o.tensor_cores == 1


@pytest.mark.parametrize("ov", [1, 2, 3])
def test_host_overlap_sets_match_oracle(A, ov):
    """Sec. 2.1 sets from the library's host code equal the oracle's."""
    M = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=3, channel_value=1e3)
    part = synth.bfs_partition(M, 7, seed=3, min_size=30, max_size=140)
    As = O.to_scipy(M)
    for i in range(int(part.max()) + 1):
        I, G, D = A.overlap_sets(M.n, M.rowptr, M.colind, part, i, ov)
        oI, oG, oD = O.subdomain_sets(As, part, i, ov)
        assert np.array_equal(I, oI) and np.array_equal(G, oG) and np.array_equal(D, oD)


def test_host_overlap_sets_fixture(A):
    """The hand-derived 4x4-grid sets of tests/golden (Sec. 2.1)."""
    M = synth.laplace2d(4)
    part = synth.box_partition_2d(4, 2)
    I, G, D = A.overlap_sets(M.n, M.rowptr, M.colind, part, 0, 1)
    assert list(I) == [0, 1, 4, 5] and list(G) == [2, 6, 8, 9] and list(D) == [3, 7, 10, 12, 13]


def test_host_overlap_sets_rejects_bad_graph(A):
    M = synth.laplace2d(4)
    bad = M.colind.copy()
    bad[3] = 99
    with pytest.raises(A.AmddError):
        A.overlap_sets(M.n, M.rowptr, bad, synth.box_partition_2d(4, 2), 0, 1)


@pytest.mark.parametrize("tau", [0.5, 100.0])
def test_host_lanczos_extremes_match_oracle(A, tau):
    """The library's Lanczos condition estimate (host code) on the oracle's
    own PCG coefficients equals the oracle's dense tridiagonal eigenvalues."""
    M = synth.diffusion3d(8, sigma=1.0, corr=2.0, n_channels=2, seed=1, channel_value=1e3)
    part = synth.bfs_partition(M, 6, seed=1, min_size=40, max_size=160)
    S = O.setup(M, part, int(part.max()) + 1, 1, tau)
    co = []
    O.pcg(S.A, synth.rhs(M.n, 0), lambda r: O.apply(S, r), rtol=1e-8, coeffs=co)
    al = [v for t, v in co if t == "a"]
    be = [v for t, v in co if t == "b"][: len(al) - 1]
    lo, hi = A.lanczos_extremes(al, be)
    olo, ohi = O.lanczos_extremes(co)
    assert lo == pytest.approx(olo, rel=1e-12) and hi == pytest.approx(ohi, rel=1e-12)
    for k in (1, 2, 3):
        lo, hi = A.lanczos_extremes(al[:k], be[: k - 1])
        olo, ohi = O.lanczos_extremes([("a", a) for a in al[:k]] + [("b", b) for b in be[: k - 1]])
        assert lo == pytest.approx(olo, rel=1e-12) and hi == pytest.approx(ohi, rel=1e-12)


def test_host_lanczos_extremes_rejects_bad_input(A):
    with pytest.raises(A.AmddError):
        A.lanczos_extremes([1.0, -2.0], [0.5])
    with pytest.raises(A.AmddError):
        A.lanczos_extremes([1.0, 2.0], [-0.5])
    lo, hi = A.lanczos_extremes([], [])
    assert np.isnan(lo) and np.isnan(hi)
