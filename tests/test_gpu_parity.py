"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every bar has a fixed part and a part that scales with the FP64 rounding
envelope of the oracle itself on the same problem: the largest change of the
oracle's result when the unknowns are relabelled (three seeded permutations;
exact arithmetic is invariant to the order of Omega_i).  On well-conditioned
problems the envelope is ~1e-15 and the fixed part decides; on the layered
elasticity problems (modulus contrast 1e5, sigma_1 / sigma_min of X_i ~ 4e6)
FP64 itself fixes the small singular directions, the spans of near-degenerate
eigenvectors and the apply only to the envelope.
  * singular values of X_i: |dsigma_j| <= 1e-10 sigma_j + 20 eta_sigma;
  * eigenvalues of eq. (Zi), compared as mu = 1/lambda (ascending, mu = 0 for
    lambda = +inf): |dmu| <= 1e-8 mu + 20 eta_mu;
  * selected count p_i exactly; selected span: sine of the largest principal
    angle <= max(1e-8, 20 eta_span);
  * one apply z = M^{-1} r: 1e-10 relative, or 20 eta_apply if larger, both
    in norm and entry by entry (|z_gpu - z_o| <= bar ||z_o||_inf at every
    unknown, so an error confined to a few unknowns cannot hide in the norm);
  * PCG iterations to 1e-8: equal within +-1; PCG solutions at rtol 1e-12:
    1e-10 relative (plus 20 eta_apply), in norm and entry by entry;
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


def _elas(ne, box, layer, ov, tau):
    M, _, xyz = synth.elasticity3d(ne, layer=layer)
    part = synth.box_partition_dofs(xyz, (box, box, box))
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
    "elas6_layer2_ov1_tau0.5": lambda: _elas(6, 4, 2, 1, 0.5),
    "elas5_layer2_ov2_tau100": lambda: _elas(5, 3, 2, 2, 100.0),
}

_cache = {}


def _entrywise(zg, zo, bar):
    """Norm-wise and entry-wise agreement: every entry within bar * ||z_o||_inf."""
    assert np.linalg.norm(zg - zo) <= bar * np.linalg.norm(zo)
    err = np.abs(zg - zo)
    k = int(np.argmax(err))
    assert err[k] <= bar * np.abs(zo).max(), f"entry {k}: {zg[k]!r} vs {zo[k]!r}"


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
    eta = _envelope(name)["sigma"]
    for i, s in enumerate(S.subs):
        sg = A.get_singular_values(P.h, i)
        so = np.sort(s.sigma)[::-1]
        assert np.all(np.abs(sg - so) <= 1e-10 * so + 20 * eta[i]), f"subdomain {i}"


def _mu(lam):
    with np.errstate(divide="ignore"):
        return np.sort(np.where(np.isinf(lam), 0.0, 1.0 / lam))


_env = {}


def _span_sine(Za, Zb):
    qa, _ = np.linalg.qr(Za)
    qb, _ = np.linalg.qr(Zb)
    return np.linalg.norm(qb - qa @ (qa.T @ qb), 2)


def _envelope(name):
    """FP64 rounding envelope of the oracle on each subdomain: the largest
    change of mu, sigma (absolute), the selected span and one apply over three
    random relabellings of the unknowns (same sets, different FP64 rounding)."""
    if name not in _env:
        M, part, N, ov, tau, S, dA, dpart, P = _case(name)
        eta = {"mu": np.zeros(N), "sigma": np.zeros(N), "span": np.zeros(N), "apply": 0.0}
        r = np.random.default_rng(7).uniform(-1, 1, M.n)
        zo = O.apply(S, r)
        for seed in (101, 202, 303):
            perm = np.random.default_rng(seed).permutation(M.n)
            inv = np.argsort(perm)
            Sp = O.setup(S.A[perm][:, perm].tocsr(), np.asarray(part)[perm], N, ov, tau)
            zp = O.apply(Sp, r[perm])[inv]
            eta["apply"] = max(eta["apply"], np.linalg.norm(zp - zo) / np.linalg.norm(zo))
            for i in range(N):
                s, t = S.subs[i], Sp.subs[i]
                eta["mu"][i] = max(eta["mu"][i], np.abs(_mu(t.lam) - _mu(s.lam)).max())
                eta["sigma"][i] = max(eta["sigma"][i],
                                      np.abs(np.sort(t.sigma)[::-1] - np.sort(s.sigma)[::-1]).max())
                if 0 < s.p < len(s.I) and t.p == s.p:
                    Zo = np.zeros((M.n, s.p))
                    Zo[s.I] = s.Z[: len(s.I)]
                    Zq = np.zeros((M.n, s.p))
                    Zq[perm[t.I]] = t.Z[: len(t.I)]
                    eta["span"][i] = max(eta["span"][i], _span_sine(Zq, Zo))
        _env[name] = eta
    return _env[name]


@pytest.mark.parametrize("name", list(CASES))
def test_eigenvalues_and_selection(name):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    env = _envelope(name)
    eta = env["mu"]
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
            assert _span_sine(Zt.T, s.Z[: len(s.I)]) <= max(1e-8, 20 * env["span"][i])
        AII = s.Aii[: len(s.I), : len(s.I)]
        if 0 < s.p < len(s.I):
            # the selected eigenvectors: A_II-orthonormal rows on Omega_Ii
            G = Zt @ AII @ Zt.T
            assert np.allclose(G, np.eye(s.p), atol=1e-9)
        elif s.p == len(s.I):
            # every eigenvalue selected: the span is all of R^nI and the basis
            # is diag(A_II)^{-1/2}
            assert np.array_equal(Zt, np.diag(1.0 / np.sqrt(np.diag(AII))))


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
    bar = max(1e-10, 20 * _envelope(name)["apply"])
    _entrywise(zg, zo, bar)
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
        _entrywise(zd[k].cpu().numpy(), zo, 1e-10)


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
    bar = 1e-10 + 20 * _envelope(name)["apply"]
    _entrywise(xd2.cpu().numpy(), xo, bar)
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


@pytest.mark.parametrize("name,nrhs", [("diff8_bfs_ov1_tau0.5", 5), ("lap16_box4_tau0.5", 10)])
def test_pcg_batched_rhs(name, nrhs):
    """nrhs independent solves advanced together (batches of up to 8 share each
    SpMV and apply): every solution matches the oracle's tight solve, the first
    right-hand side's iteration count matches the oracle's, and a zero
    right-hand side returns x = 0."""
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    B = synth.rhs(M.n, 21, nrhs=nrhs)
    B[3] = 0.0
    bd = to_device(B)
    xd = torch.zeros_like(bd)
    st = P.solve(bd, xd, nrhs=nrhs, rtol=1e-12)
    assert st.converged == 1
    _, its_o, _ = O.pcg(S.A, B[0], lambda r: O.apply(S, r), rtol=1e-12)
    assert abs(st.iterations - its_o) <= 1
    X = xd.cpu().numpy()
    for k in range(nrhs):
        if k == 3:
            assert np.all(X[k] == 0.0)
            continue
        xo, _, _ = O.pcg(S.A, B[k], lambda r: O.apply(S, r), rtol=1e-12)
        _entrywise(X[k], xo, 1e-10)
    # the batched apply (one pass over the factors for up to 8 right-hand sides)
    zd = torch.empty_like(bd)
    P.apply(bd, zd, nrhs=nrhs)
    for k in (0, nrhs - 1):
        zo = O.apply(S, B[k])
        _entrywise(zd[k].cpu().numpy(), zo, 1e-10)


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


@pytest.mark.parametrize("where", ["A_nan", "A_inf", "b_nan", "b_inf", "x0_nan"])
def test_nonfinite_inputs_are_rejected(where):
    """A NaN or an infinity in A (amdd_setup), in b or in the initial guess
    (amdd_pcg_solve, amdd_gmres_solve) is AMDD_ERR_INVALID, not a garbage
    solve."""
    M = synth.laplace2d(12)
    part = torch.from_numpy(synth.box_partition_2d(12, 6)).cuda()
    bad = np.nan if where.endswith("nan") else np.inf
    if where.startswith("A"):
        val = M.val.copy()
        val[17] = bad
        with pytest.raises(A.AmddError) as e:
            Preconditioner(DeviceMatrix(synth.CSR(M.n, M.rowptr, M.colind, val)), part, 4, 1, 50.0)
        assert e.value.status == 1
        return
    P = Preconditioner(DeviceMatrix(M), part, 4, 1, 50.0)
    try:
        b = synth.rhs(M.n, 1)
        x0 = np.zeros(M.n)
        (x0 if where == "x0_nan" else b)[5] = bad
        bd, xd = to_device(b), to_device(x0)
        with pytest.raises(A.AmddError) as e:
            P.solve(bd, xd, rtol=1e-8)
        assert e.value.status == 1
        with pytest.raises(A.AmddError) as e:
            P.gmres(bd, xd)
        assert e.value.status == 1
        # the handle stays usable
        st = P.solve(to_device(synth.rhs(M.n, 1)), torch.zeros_like(bd), rtol=1e-8)
        assert st.converged == 1
    finally:
        P.close()


@pytest.mark.parametrize("name", ["lap64_box16_tau50_C1", "diff8_bfs_ov1_tau0.5", "lap18_box6_ov2_tau0.5"])
def test_pcg_graph_equals_launches(name):
    """use_graphs = 1 replays the PCG iterations as one CUDA graph (a device
    while-loop); use_graphs = 0 launches them one by one.  Same kernels, same
    order: the same iteration count, the same bits of x and the same Lanczos
    estimate."""
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    o = A.opts_default()
    o.use_graphs = 0
    Pn = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        b = to_device(synth.rhs(M.n, 5))
        xg, xn = torch.zeros_like(b), torch.zeros_like(b)
        sg = P.solve(b, xg, rtol=1e-8)
        sn = Pn.solve(b, xn, rtol=1e-8)
        assert P.info().graph_solves >= 1 and Pn.info().graph_solves == 0
        assert sg.iterations == sn.iterations and sg.converged == sn.converged == 1
        assert torch.equal(xg, xn)
        assert sg.rel_residual == sn.rel_residual and sg.true_rel_residual == sn.true_rel_residual
        assert sg.cond_est == sn.cond_est
        # a second solve on the same handle reuses the graph; maxit stops it
        with pytest.raises(A.AmddError) as e:
            P.solve(b, torch.zeros_like(b), rtol=1e-14, maxit=3)
        assert e.value.status == 3
        x3n = torch.zeros_like(b)
        with pytest.raises(A.AmddError):
            Pn.solve(b, x3n, rtol=1e-14, maxit=3)
        x3g = torch.zeros_like(b)
        st = A.pcg_solve(P.h, b.data_ptr(), x3g.data_ptr(), 1, 1e-14, 3, allow_noconv=True)
        assert st.iterations == 3 and torch.equal(x3g, x3n)
    finally:
        Pn.close()


def test_memory_budget():
    """mem_budget: a setup that needs more device memory than the budget fails
    with AMDD_ERR_OOM before allocating past it; a budget equal to what the
    same setup reported as its peak suffices."""
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap16_box4_tau0.5")
    peak = P.info().device_bytes_peak
    assert peak > 0
    o = A.opts_default()
    o.mem_budget = peak // 2
    with pytest.raises(A.AmddError) as e:
        Preconditioner(dA, dpart, N, ov, tau, o)
    assert e.value.status == 4
    o.mem_budget = peak
    Q = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        assert Q.info().n_C == S.nC and Q.info().device_bytes_peak <= peak
    finally:
        Q.close()


def test_tie_band_counts_threshold_eigenvalues():
    """One subdomain: every eigenvalue of eq. (Zi) is a_j / (a_j + sigma_1 eps),
    within 1e-13 of 1.  With tau = 1 all of them lie in the default band
    |lambda tau - 1| <= 1e-10 and are counted; in exact arithmetic none is
    selected (lambda < 1), but rounding at the 1e-16 level decides each one,
    so any count is a correct selection there.  With tau = 2 none is near the
    threshold 1/2 and all are selected."""
    M = synth.laplace2d(12)
    dA = DeviceMatrix(M)
    part = torch.zeros(M.n, dtype=torch.int32, device="cuda")
    for tau, tied in ((1.0, M.n), (2.0, 0)):
        Q = Preconditioner(dA, part, 1, 1, tau)
        try:
            assert Q.info().n_tied == tied, (tau, Q.info().n_tied)
            if tau == 2.0:
                assert Q.info().n_C == M.n
        finally:
            Q.close()


@pytest.mark.parametrize("name", ["diff8_bfs_ov1_tau0.5", "lap18_box6_ov2_tau0.5"])
def test_gemm_autotuner_changes_no_bits(name):
    """The GEMM tile autotuner (autotune = 1, the default) measures tile sizes
    per size bucket; every tile size sums each output over k in the same
    order, so a handle set up without it gives the same bits: eigenvalues,
    singular values and one apply."""
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    assert P.info().tuned_buckets >= 1
    o = A.opts_default()
    o.autotune = 0
    Q = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        for i in range(N):
            assert np.array_equal(A.get_eigenvalues(P.h, i), A.get_eigenvalues(Q.h, i))
            assert np.array_equal(A.get_singular_values(P.h, i), A.get_singular_values(Q.h, i))
        rd = to_device(synth.rhs(M.n, 8))
        z1, z2 = torch.empty_like(rd), torch.empty_like(rd)
        P.apply(rd, z1)
        Q.apply(rd, z2)
        assert torch.equal(z1, z2)
    finally:
        Q.close()


@pytest.mark.parametrize("name", ["lap16_box4_tau0.5", "lap64_box16_tau50_C1", "diff8_bfs_ov1_tau0.5",
                                  "diff9_bfs_ov2_tau100", "elas6_layer2_ov1_tau0.5"])
def test_sparse_local_factors(name):
    """local_solver = 1: the local solves use sparse Cholesky factors of the
    A_ii in a nested-dissection order (Sec. 4.1's exact local Cholesky, with
    the symbolic fill only).  One apply equals the oracle's within the bars of
    test_apply_matches_oracle, entry by entry, and is bitwise reproducible; the
    batched apply and PCG agree with the oracle; the factors hold fewer entries
    than the dense triangles."""
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    o = A.opts_default()
    o.local_solver = 1
    Q = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        info = Q.info()
        dense = sum(len(s.omega) * (len(s.omega) + 1) // 2 for s in S.subs)
        assert 0 < info.sparse_local_nnz < dense
        rng = np.random.default_rng(7)
        r = rng.uniform(-1, 1, M.n)
        zo = O.apply(S, r)
        rd = to_device(r)
        z1, z2 = torch.empty_like(rd), torch.empty_like(rd)
        Q.apply(rd, z1)
        Q.apply(rd, z2)
        assert torch.equal(z1, z2)
        bar = max(1e-10, 20 * _envelope(name)["apply"])
        _entrywise(z1.cpu().numpy(), zo, bar)
        R = synth.rhs(M.n, 11, nrhs=3)
        Rd = to_device(R)
        Zd = torch.empty_like(Rd)
        Q.apply(Rd, Zd, nrhs=3)
        for k in range(3):
            _entrywise(Zd[k].cpu().numpy(), O.apply(S, R[k]), bar)
        b = synth.rhs(M.n, 0)
        _, its_o, _ = O.pcg(S.A, b, lambda v: O.apply(S, v), rtol=1e-8)
        bd = to_device(b)
        x = torch.zeros_like(bd)
        st = Q.solve(bd, x, rtol=1e-8)
        assert st.converged == 1 and abs(st.iterations - its_o) <= 1 and st.true_rel_residual <= 1.5e-8
    finally:
        Q.close()


def test_sparse_local_factors_mixed_and_auto():
    """The mixed form with sparse FP32 factors reaches 1e-8 with the dense
    mixed form's iteration count +-1; local_solver = 2 keeps the sparse factors
    on 16 x 16 boxes (a few per cent of the dense triangles)."""
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap64_box16_tau50_C1")
    b = to_device(synth.rhs(M.n, 0))
    its = {}
    for ls in (0, 1, 2):
        o = A.opts_default()
        o.precision = 1
        o.local_solver = ls
        Q = Preconditioner(dA, dpart, N, ov, tau, o)
        try:
            x = torch.zeros_like(b)
            st = Q.solve(b, x, rtol=1e-8)
            assert st.converged == 1 and st.true_rel_residual <= 2e-8
            its[ls] = st.iterations
            if ls:
                assert Q.info().sparse_local_nnz > 0
        finally:
            Q.close()
    assert abs(its[1] - its[0]) <= 1 and its[2] == its[1]
