"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (FP64 throughout):
  * singular values of X_i: 1e-10 relative;
  * eigenvalues of eq. (Zi), compared as mu = 1/lambda (ascending, mu = 0 for
    lambda = +inf): |mu_gpu - mu_oracle| <= 1e-8 mu_oracle + 20 eta_i, where
    eta_i is the FP64 rounding envelope of the oracle itself on subdomain i:
    the largest change of its mu when the unknowns are relabelled (two random
    permutations; exact arithmetic is invariant to the order of Omega_i).  On
    well-conditioned problems eta ~ 1e-15, so the bar is 1e-8 relative; on
    high-contrast ones it widens only where FP64 cannot fix mu (the range
    between the finite modes and the eps-cluster);
  * selected count p_i exactly; selected span to 1e-8 (sine of the largest
    principal angle);
  * one apply z = M^{-1} r: 1e-10 relative (2-norm);
  * PCG iterations to 1e-8: equal within +-1; PCG solutions at rtol 1e-12:
    1e-10 relative;
  * bitwise run-to-run reproducibility of apply and PCG (deterministic
    reductions).
"""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, Preconditioner, to_device  # noqa: E402


def _lap(m, box, ov, tau):
    M = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    return M, part, int(part.max()) + 1, ov, tau


def _diff(m, N, seed, ov, tau, lo, hi, cv=1e3, sigma=1.0):
    M = synth.diffusion3d(m, sigma=sigma, corr=2.0, n_channels=2, seed=seed, channel_value=cv)
    part = synth.bfs_partition(M, N, seed=seed, min_size=lo, max_size=hi)
    return M, part, int(part.max()) + 1, ov, tau


CASES = {
    "lap16_box4_tau50": lambda: _lap(16, 4, 1, 50.0),
    "lap16_box4_tau0.5": lambda: _lap(16, 4, 1, 0.5),
    "lap18_box6_ov2_tau0.5": lambda: _lap(18, 6, 2, 0.5),
    "lap64_box16_tau50_C1": lambda: _lap(64, 16, 1, 50.0),
    "diff8_bfs_ov1_tau0.5": lambda: _diff(8, 6, 1, 1, 0.5, 40, 160),
    "diff9_bfs_ov2_tau100": lambda: _diff(9, 5, 2, 2, 100.0, 60, 220),
    "diff10_bfs_ov1_tau0.1_contrast": lambda: _diff(10, 8, 4, 1, 0.1, 60, 200, cv=1e5, sigma=1.5),
    "single_subdomain": lambda: (synth.laplace2d(12), np.zeros(144, np.int32), 1, 1, 50.0),
}

_cache = {}


def _case(name):
    if name not in _cache:
        M, part, N, ov, tau = CASES[name]()
        S = O.setup(M, part, N, ov, tau)
        dA = DeviceMatrix(M)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        P = Preconditioner(dA, dpart, N, ov, tau)
        _cache[name] = (M, part, N, ov, tau, S, dA, dpart, P)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_sizes_match(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    for i, s in enumerate(S.subs):
        nI, nG, nD, p = A.get_subdomain(P.h, i)
        assert (nI, nG, nD) == (len(s.I), len(s.G), len(s.D))
        assert p == s.p
    assert P.info().n_C == S.nC


@pytest.mark.parametrize("name", list(CASES))
def test_singular_values(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    for i, s in enumerate(S.subs):
        sg = A.get_singular_values(P.h, i)
        assert np.allclose(sg, s.sigma, rtol=1e-10, atol=0)


def _mu(lam):
    with np.errstate(divide="ignore"):
        return np.sort(np.where(np.isinf(lam), 0.0, 1.0 / lam))


_env = {}


def _envelope(name):
    """eta_i: largest change of the oracle's mu on subdomain i over two random
    relabellings of the unknowns (same sets, different FP64 rounding)."""
    if name not in _env:
        M, part, N, ov, tau, S, dA, dpart, P = _case(name)
        eta = np.zeros(N)
        for seed in (101, 202):
            perm = np.random.default_rng(seed).permutation(M.n)
            Sp = O.setup(S.A[perm][:, perm].tocsr(), np.asarray(part)[perm], N, ov, tau)
            for i in range(N):
                eta[i] = max(eta[i], np.abs(_mu(Sp.subs[i].lam) - _mu(S.subs[i].lam)).max())
        _env[name] = eta
    return _env[name]


@pytest.mark.parametrize("name", list(CASES))
def test_eigenvalues_and_selection(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    eta = _envelope(name)
    for i, s in enumerate(S.subs):
        lg = A.get_eigenvalues(P.h, i)
        assert len(lg) == len(s.lam)
        mo, mg = _mu(s.lam), _mu(lg)
        bar = 1e-8 * mo + 20 * eta[i]
        worst = np.max(np.abs(mg - mo) / bar)
        assert worst <= 1.0, f"subdomain {i}: |dmu|/bar = {worst:.2f} (eta {eta[i]:.2e})"
        Zt = A.get_coarse_block(P.h, i)
        assert Zt.shape[0] == s.p
        if 0 < s.p < len(s.I):
            q1, _ = np.linalg.qr(Zt.T)
            q2, _ = np.linalg.qr(s.Z[: len(s.I)])
            assert np.linalg.norm(q2 - q1 @ (q1.T @ q2), 2) < 1e-8
        if s.p:
            # A_II-orthonormal columns on Omega_Ii
            AII = s.Aii[: len(s.I), : len(s.I)]
            G = Zt @ AII @ Zt.T
            assert np.allclose(G, np.eye(s.p), atol=1e-9)


@pytest.mark.parametrize("name", list(CASES))
def test_apply_matches_oracle(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    rng = np.random.default_rng(7)
    r = rng.uniform(-1, 1, M.n)
    zo = O.apply(S, r)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P.apply(rd, zd)
    zg = zd.cpu().numpy()
    assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)
    z2 = torch.empty_like(rd)
    P.apply(rd, z2)
    assert torch.equal(zd, z2), "apply is not bitwise reproducible"


def test_apply_multiple_rhs():
    M, part, N, ov, tau, S, dA, dpart, P = _case("diff8_bfs_ov1_tau0.5")
    R = synth.rhs(M.n, 11, nrhs=3)
    rd = to_device(R)
    zd = torch.empty_like(rd)
    P.apply(rd, zd, nrhs=3)
    for k in range(3):
        zo = O.apply(S, R[k])
        assert np.linalg.norm(zd[k].cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_matches_oracle(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    b = synth.rhs(M.n, 0)
    _, its_o, hist = O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-8)
    bd = to_device(b)
    xd = torch.zeros_like(bd)
    st = P.solve(bd, xd, rtol=1e-8)
    assert st.converged == 1
    assert abs(st.iterations - its_o) <= 1
    assert st.true_rel_residual <= 1.5e-8
    # tight solve: solutions agree to 1e-10
    xo, _, _ = O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-12)
    xd2 = torch.zeros_like(bd)
    P.solve(bd, xd2, rtol=1e-12)
    assert np.linalg.norm(xd2.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
    xd3 = torch.zeros_like(bd)
    P.solve(bd, xd3, rtol=1e-12)
    assert torch.equal(xd2, xd3), "PCG is not bitwise reproducible"


@pytest.mark.parametrize("name", ["lap16_box4_tau0.5", "diff8_bfs_ov1_tau0.5", "diff9_bfs_ov2_tau100"])
def test_condition_estimate(name):
    """The Lanczos condition estimate of the GPU PCG equals the oracle's on the
    same iterations (1e-6), lies inside the dense spectrum of M^{-1} A and
    under the bound of Sec. 3.2."""
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    b = synth.rhs(M.n, 0)
    co = []
    _, its_o, _ = O.pcg(S.A, b, lambda r: O.apply(S, r), rtol=1e-8, coeffs=co)
    bd = to_device(b)
    xd = torch.zeros_like(bd)
    st = P.solve(bd, xd, rtol=1e-8)
    lo, hi = O.lanczos_extremes(co)
    if st.iterations == its_o:
        assert st.ritz_min == pytest.approx(lo, rel=1e-6) and st.ritz_max == pytest.approx(hi, rel=1e-6)
    Minv = np.column_stack([O.apply(S, e) for e in np.eye(M.n)])
    ev = np.sort(np.linalg.eigvals(Minv @ S.A.toarray()).real)
    assert ev[0] * (1 - 1e-8) <= st.ritz_min and st.ritz_max <= ev[-1] * (1 + 1e-8)
    bound = O.condition_bound(O.colouring_number(S), O.splitting_constant(S), tau)
    assert st.cond_est == pytest.approx(st.ritz_max / st.ritz_min) and st.cond_est <= bound


def test_pcg_initial_guess_and_zero_rhs():
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap16_box4_tau0.5")
    b = synth.rhs(M.n, 2)
    xs = np.linalg.solve(S.A.toarray(), b)
    bd = to_device(b)
    x0 = to_device(xs)  # exact initial guess: converged at once
    st = P.solve(bd, x0, rtol=1e-8)
    assert st.iterations == 0 and st.converged == 1
    z = torch.zeros_like(bd)
    x = torch.ones_like(bd)
    st = P.solve(z, x, rtol=1e-8)
    assert st.converged == 1 and float(x.abs().max()) == 0.0


def test_pcg_maxit_reports_noconv():
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap16_box4_tau0.5")
    bd = to_device(synth.rhs(M.n, 4))
    x = torch.zeros_like(bd)
    with pytest.raises(A.AmddError) as e:
        P.solve(bd, x, rtol=1e-14, maxit=2)
    assert e.value.status == 3


@pytest.mark.parametrize("m,seed", [(37, 0), (5, 1), (64, 2)])
def test_spmv_matches_scipy(m, seed):
    M = synth.laplace2d(m) if seed != 2 else synth.diffusion3d(16, seed=2, n_channels=3)
    dA = DeviceMatrix(M)
    x = np.random.default_rng(seed).standard_normal(M.n)
    xd = to_device(x)
    yd = torch.empty_like(xd)
    A.spmv(dA.csr, xd.data_ptr(), yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    yo = O.to_scipy(M) @ x
    assert np.allclose(yd.cpu().numpy(), yo, rtol=1e-14, atol=1e-14 * np.abs(yo).max())


def test_not_spd_is_reported():
    M = synth.laplace2d(12)
    val = M.val.copy()
    d0 = np.flatnonzero((M.colind == 5) & (np.repeat(np.arange(M.n), np.diff(M.rowptr)) == 5))[0]
    val[d0] = -4.0
    Mb = synth.CSR(M.n, M.rowptr, M.colind, val)
    dA = DeviceMatrix(Mb)
    part = torch.from_numpy(synth.box_partition_2d(12, 6)).cuda()
    with pytest.raises(A.AmddError) as e:
        Preconditioner(dA, part, 4, 1, 50.0)
    assert e.value.status == 2


def test_invalid_partitions_are_rejected():
    M = synth.laplace2d(8)
    dA = DeviceMatrix(M)
    part = synth.box_partition_2d(8, 4)
    with pytest.raises(A.AmddError) as e:  # subdomain 4 empty
        Preconditioner(dA, torch.from_numpy(part).cuda(), 5, 1, 50.0)
    assert e.value.status == 1
    bad = part.copy()
    bad[3] = 7
    with pytest.raises(A.AmddError) as e:
        Preconditioner(dA, torch.from_numpy(bad).cuda(), 4, 1, 50.0)
    assert e.value.status == 1
    with pytest.raises(A.AmddError):
        Preconditioner(dA, torch.from_numpy(part).cuda(), 4, 0, 50.0)
    with pytest.raises(A.AmddError):
        Preconditioner(dA, torch.from_numpy(part).cuda(), 4, 1, -1.0)
