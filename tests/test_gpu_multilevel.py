"""Parity of the multilevel form (Sec. 3.2, last paragraph; Sec. 4.2) through
the C ABI with the FP64 CPU oracle (oracle/multilevel.py).

The library's coarse basis differs from the oracle's by an orthogonal matrix
per subdomain (both are A_II-orthonormal bases of the same span), so its E
is a block-orthogonal congruence of the oracle's.  The second-level
construction commutes with that congruence (pinned on the CPU by
test_orthogonal_coarse_basis_invariance), and so do GMRES iterates.  Bars:
  * second-level sizes and selections p_i equal the oracle's; second-level
    eigenvalues of eq. (Zi) (invariant under the congruence) as at the first
    level: |dmu| <= 1e-8 mu + 20 eta_i, eta_i the oracle's own FP64 rounding
    envelope (largest change of its mu under three relabellings of E's
    unknowns; between mu ~ 1e-8 and 1e-4 two FP64 evaluations of this pencil
    differ by percents);
  * with a tight inner tolerance one application equals the two-level
    deflated application to 1e-9 relative;
  * with the paper's inner GMRES(30) to 1e-4 one application equals the
    oracle's multilevel application to 1e-6 relative (the inner solve stops
    at the same step), and the outer flexible GMRES(30) reaches 1e-8 in the
    oracle's outer iteration count +-1.
"""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import multilevel as ML

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, to_device  # noqa: E402


def _lap(m, box, g, tau, tau2, ov=1, ov2=1):
    M = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    nb = m // box
    groups = synth.box_groups_2d(nb, g)
    return M, part, nb * nb, ov, tau, groups, int(groups.max()) + 1, ov2, tau2


def _diff(tau, tau2, N2):
    M = synth.diffusion3d(10, sigma=1.0, corr=2.0, n_channels=2, seed=2, channel_value=1e3)
    part = synth.bfs_partition(M, 10, seed=2, min_size=50, max_size=180)
    N = int(part.max()) + 1
    groups = (np.arange(N) * N2 // N).astype(np.int32)
    return M, part, N, 1, tau, groups, N2, 1, tau2


CASES = {
    "lap24_box6_g2_tau0.5": lambda: _lap(24, 6, 2, 0.5, 0.5),
    "lap32_box4_g4_tau0.5_ov2": lambda: _lap(32, 4, 4, 0.5, 0.5, ov2=2),
    "diff10_bfs_g3_tau0.5": lambda: _diff(0.5, 0.5, 3),
}

_cache = {}


class _Level:
    def __init__(self, M, part, N, ov, tau, groups, N2, ov2, tau2, inner_rtol=1e-4):
        self.dA = DeviceMatrix(M)
        self.dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        o = A.opts_default()
        o.keep_coarse_matrix = 1
        self.h = A.setup(self.dA.csr, self.dpart.data_ptr(), N, ov, tau, o, torch.cuda.current_stream().cuda_stream)
        self.h2 = A.setup_next_level(self.h, groups, N2, ov2, tau2, None, 30, inner_rtol, 100)

    def close(self):
        A.destroy(self.h)


def _case(name):
    if name not in _cache:
        M, part, N, ov, tau, groups, N2, ov2, tau2 = CASES[name]()
        ml = ML.setup(M, part, N, ov, tau, groups, N2, ov2, tau2)
        ml_groups[id(ml)] = groups
        _cache[name] = (M, part, N, ov, tau, groups, N2, ov2, tau2, ml, _Level(M, part, N, ov, tau, groups, N2,
                                                                                 ov2, tau2))
    return _cache[name]


def _envelope2(ml, N2, ov2, tau2):
    """FP64 rounding envelope of the oracle's second level: the largest change
    of each subdomain's mu under three seeded relabellings of E's unknowns
    (exact arithmetic is invariant to that order)."""
    E, p2 = ml.E, ML.coarse_partition(ml.S1, ml_groups[id(ml)])
    eta = np.zeros(N2)
    for seed in (101, 202, 303):
        perm = np.random.default_rng(seed).permutation(E.shape[0])
        Sp = O.setup(E[perm][:, perm].tocsr(), p2[perm], N2, ov2, tau2)
        for i in range(N2):
            eta[i] = max(eta[i], np.abs(_mu(Sp.subs[i].lam) - _mu(ml.S2.subs[i].lam)).max())
    return eta


ml_groups = {}


def _mu(lam):
    with np.errstate(divide="ignore"):
        return np.sort(np.where(np.isinf(lam), 0.0, 1.0 / lam))


@pytest.mark.parametrize("name", list(CASES))
def test_second_level_sizes_and_eigenvalues(name):
    M, part, N, ov, tau, groups, N2, ov2, tau2, ml, L = _case(name)
    info = A.get_info(L.h)
    assert info.levels == 2 and info.n_C == ml.S1.nC
    i2 = A.get_info(L.h2)
    assert i2.n == ml.S1.nC and i2.N == N2 and i2.n_C == ml.S2.nC
    eta = _envelope2(ml, N2, ov2, tau2)
    for i, s in enumerate(ml.S2.subs):
        nI, nG, nD, p = A.get_subdomain(L.h2, i)
        assert (nI, nG, nD, p) == (len(s.I), len(s.G), len(s.D), s.p)
        mg, mo = _mu(A.get_eigenvalues(L.h2, i)), _mu(s.lam)
        assert np.all(np.abs(mg - mo) <= 1e-8 * mo + 20 * eta[i]), f"second-level subdomain {i} (eta {eta[i]:.2e})"


@pytest.mark.parametrize("name", list(CASES))
def test_apply_with_exact_inner_solve_is_two_level(name):
    M, part, N, ov, tau, groups, N2, ov2, tau2, ml, _ = _case(name)
    L = _Level(M, part, N, ov, tau, groups, N2, ov2, tau2, inner_rtol=1e-13)
    try:
        r = np.random.default_rng(7).uniform(-1, 1, M.n)
        rd = to_device(r)
        zd = torch.empty_like(rd)
        A.apply_form(L.h, A.FORM_DEFLATED, rd.data_ptr(), zd.data_ptr())
        zo = O.apply_deflated(ml.S1, r)
        assert np.linalg.norm(zd.cpu().numpy() - zo) <= 1e-9 * np.linalg.norm(zo)
        info = A.get_info(L.h)
        assert info.inner_solves == 1 and info.inner_iterations >= 1
    finally:
        L.close()


@pytest.mark.parametrize("name", list(CASES))
def test_apply_with_inexact_inner_solve_matches_oracle(name):
    M, part, N, ov, tau, groups, N2, ov2, tau2, ml, L = _case(name)
    r = np.random.default_rng(8).uniform(-1, 1, M.n)
    ml.inner_its.clear()
    zo = ML.apply_deflated(ml, r)
    before = A.get_info(L.h)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    A.apply_form(L.h, A.FORM_DEFLATED, rd.data_ptr(), zd.data_ptr())
    after = A.get_info(L.h)
    its_gpu = after.inner_iterations - before.inner_iterations
    assert its_gpu == ml.inner_its[-1], (its_gpu, ml.inner_its)
    assert np.linalg.norm(zd.cpu().numpy() - zo) <= 1e-6 * np.linalg.norm(zo)
    # the additive form uses the same inexact coarse solve
    zd2 = torch.empty_like(rd)
    A.apply(L.h, rd.data_ptr(), zd2.data_ptr(), 1)
    c = ml.S1.W.T @ r
    e = ML.coarse_solve(ml, c)
    za = ml.S1.W @ e + O.apply_one_level(ml.S1, r)
    assert np.linalg.norm(zd2.cpu().numpy() - za) <= 1e-6 * np.linalg.norm(za)


@pytest.mark.parametrize("name", list(CASES))
def test_three_level_fgmres_matches_oracle(name):
    """Outer flexible GMRES(30) to 1e-8 (Sec. 4.2): iterations +-1 of the
    oracle's, true residual 1.5e-8, and at most one more outer iteration than
    the two-level method with the exact coarse solve."""
    M, part, N, ov, tau, groups, N2, ov2, tau2, ml, L = _case(name)
    b = synth.rhs(M.n, 0)
    _, its_o, _ = ML.solve(ml, b)
    _, its_2, _ = O.gmres(ml.S1.A, b, lambda v: O.apply_deflated(ml.S1, v), restart=30, rtol=1e-8)
    bd = to_device(b)
    xd = torch.zeros_like(bd)
    st = A.gmres_solve(L.h, A.FORM_DEFLATED, bd.data_ptr(), xd.data_ptr(), 1, 30, 1e-8, 200)
    assert st.converged == 1
    assert abs(st.iterations - its_o) <= 1, (st.iterations, its_o)
    assert st.iterations <= its_2 + 1, (st.iterations, its_2)
    x = xd.cpu().numpy()
    assert np.linalg.norm(b - ml.S1.A @ x) <= 1.5e-8 * np.linalg.norm(b)
    assert A.get_info(L.h).inner_iterations_max <= 30


def test_pcg_and_batched_apply_with_next_level():
    """The batched apply runs the inexact coarse solve per right-hand side;
    PCG with the (now slightly variable) additive form still converges."""
    M, part, N, ov, tau, groups, N2, ov2, tau2, ml, L = _case("lap24_box6_g2_tau0.5")
    R = synth.rhs(M.n, 3, nrhs=2)
    Rd = to_device(R)
    Z = torch.empty_like(Rd)
    A.apply(L.h, Rd.data_ptr(), Z.data_ptr(), 2)
    for k in range(2):
        z1 = torch.empty(M.n, dtype=torch.float64, device="cuda")
        A.apply(L.h, Rd[k].data_ptr(), z1.data_ptr(), 1)
        assert torch.equal(z1, Z[k])
    b = to_device(synth.rhs(M.n, 1))
    x = torch.zeros_like(b)
    st = A.pcg_solve(L.h, b.data_ptr(), x.data_ptr(), 1, 1e-8, 300)
    assert st.converged == 1 and st.true_rel_residual <= 1.5e-8


def test_next_level_errors():
    M, part, N, ov, tau, groups, N2, ov2, tau2 = CASES["lap24_box6_g2_tau0.5"]()
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    sp = torch.cuda.current_stream().cuda_stream
    h = A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, None, sp)  # E not kept
    try:
        with pytest.raises(A.AmddError) as e:
            A.setup_next_level(h, groups, N2, ov2, tau2)
        assert e.value.status == 1
        assert A.next_level(h) is None
    finally:
        A.destroy(h)
    o = A.opts_default()
    o.keep_coarse_matrix = 1
    h = A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, o, sp)
    try:
        bad = groups.copy()
        bad[0] = N2  # out of range
        with pytest.raises(A.AmddError):
            A.setup_next_level(h, bad, N2, ov2, tau2)
        with pytest.raises(A.AmddError):  # an empty group
            A.setup_next_level(h, groups, N2 + 1, ov2, tau2)
        with pytest.raises(A.AmddError):
            A.setup_next_level(h, groups, N2, ov2, tau2, inner_restart=0)
        h2 = A.setup_next_level(h, groups, N2, ov2, tau2)
        assert h2 and A.get_info(h).levels == 2
    finally:
        A.destroy(h)
