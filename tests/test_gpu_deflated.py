"""Parity of the deflated two-level preconditioner, the one-level restricted
and additive Schwarz methods (Sec. 4.1) and right-preconditioned GMRES(m)
(through the C ABI) with the FP64 CPU oracle.

Bars:
  * one application z = M r of each form: 1e-10 relative, or 20x the
    oracle's own FP64 rounding envelope on the problem (largest change of its
    result under three seeded relabellings of the unknowns) if larger;
  * GMRES iterations to 1e-8: equal to the oracle's within +-1 (same
    restart); GMRES solutions at rtol 1e-12 agree to 1e-10 relative (plus
    the envelope); the true residual at exit is within 1.5x the tolerance;
  * bitwise run-to-run reproducibility (fixed-order reductions).
The GPU orthogonalises the Arnoldi basis with classical Gram-Schmidt applied
twice, the oracle with modified Gram-Schmidt: equal in exact arithmetic.
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
    "lap16_box4_tau0.5": lambda: _lap(16, 4, 1, 0.5),
    "lap16_box4_tau50": lambda: _lap(16, 4, 1, 50.0),
    "lap18_box6_ov2_tau0.5": lambda: _lap(18, 6, 2, 0.5),
    "lap32_box8_tau1e-12": lambda: _lap(32, 8, 1, 1e-12),
    "diff8_bfs_ov1_tau0.5": lambda: _diff(8, 6, 1, 1, 0.5, 40, 160),
    "diff10_bfs_ov1_tau0.1_contrast": lambda: _diff(10, 8, 4, 1, 0.1, 60, 200, cv=1e5, sigma=1.5),
    "single_subdomain": lambda: (synth.laplace2d(12), np.zeros(144, np.int32), 1, 1, 50.0),
    "elas5_layer2_ov1_tau0.5": lambda: _elas(5, 3, 2, 1, 0.5),
}

FORMS = {
    A.FORM_ADDITIVE: O.apply,
    A.FORM_DEFLATED: O.apply_deflated,
    A.FORM_RAS: O.apply_ras,
    A.FORM_ASM: O.apply_one_level,
}

_cache = {}
_env = {}


def _case(name):
    if name not in _cache:
        M, part, N, ov, tau = CASES[name]()
        S = O.setup(M, part, N, ov, tau)
        dA = DeviceMatrix(M)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        P = Preconditioner(dA, dpart, N, ov, tau)
        _cache[name] = (M, part, N, ov, tau, S, dA, dpart, P)
    return _cache[name]


def _envelope(name, form):
    """Largest relative change of the oracle's z = M r (form) under three
    seeded relabellings of the unknowns."""
    key = (name, form)
    if key not in _env:
        M, part, N, ov, tau, S, dA, dpart, P = _case(name)
        r = np.random.default_rng(7).uniform(-1, 1, M.n)
        zo = FORMS[form](S, r)
        eta = 0.0
        for seed in (101, 202, 303):
            perm = np.random.default_rng(seed).permutation(M.n)
            inv = np.argsort(perm)
            Sp = O.setup(S.A[perm][:, perm].tocsr(), np.asarray(part)[perm], N, ov, tau)
            zp = FORMS[form](Sp, r[perm])[inv]
            eta = max(eta, np.linalg.norm(zp - zo) / np.linalg.norm(zo))
        _env[key] = eta
    return _env[key]


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("name", list(CASES))
def test_apply_forms_match_oracle(name, form):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    r = np.random.default_rng(7).uniform(-1, 1, M.n)
    zo = FORMS[form](S, r)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P.apply_form(form, rd, zd)
    err = np.linalg.norm(zd.cpu().numpy() - zo) / np.linalg.norm(zo)
    bar = max(1e-10, 20 * _envelope(name, form))
    assert err <= bar, f"{err:.3e} > {bar:.3e}"
    z2 = torch.empty_like(rd)
    P.apply_form(form, rd, z2)
    assert torch.equal(zd, z2), "not bitwise reproducible"


def test_apply_form_additive_equals_apply():
    M, part, N, ov, tau, S, dA, dpart, P = _case("diff8_bfs_ov1_tau0.5")
    R = synth.rhs(M.n, 5, nrhs=3)
    rd = to_device(R)
    z1, z2 = torch.empty_like(rd), torch.empty_like(rd)
    P.apply(rd, z1, nrhs=3)
    P.apply_form(A.FORM_ADDITIVE, rd, z2, nrhs=3)
    assert torch.equal(z1, z2)


def test_apply_forms_several_vectors():
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap18_box6_ov2_tau0.5")
    R = synth.rhs(M.n, 9, nrhs=3)
    rd = to_device(R)
    zd = torch.empty_like(rd)
    P.apply_form(A.FORM_DEFLATED, rd, zd, nrhs=3)
    for k in range(3):
        zo = O.apply_deflated(S, R[k])
        assert np.linalg.norm(zd[k].cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)


def _gmres_pair(name, form, restart, rtol=1e-8, maxit=400, seed=0):
    M, part, N, ov, tau, S, dA, dpart, P = _case(name)
    b = synth.rhs(M.n, seed)
    xo, its_o, hist = O.gmres(S.A, b, lambda v: FORMS[form](S, v), restart=restart, rtol=rtol, maxit=maxit)
    bd = to_device(b)
    xd = torch.zeros_like(bd)
    st = P.gmres(bd, xd, form=form, restart=restart, rtol=rtol, maxit=maxit)
    return M, S, b, xo, its_o, hist, xd, st


# (case, form, restart): deflated GMRES(30) as in the experiments of Sec. 4.1,
# short restarts that take several cycles, and restart 40 with one-level
# methods whose 30-38 steps fill more than one 32-vector block of the fused
# Gram-Schmidt passes
GMRES_CASES = [(n, A.FORM_DEFLATED, 30) for n in CASES] + [
    ("lap16_box4_tau0.5", A.FORM_ADDITIVE, 30),
    ("diff8_bfs_ov1_tau0.5", A.FORM_ADDITIVE, 5),
    ("diff10_bfs_ov1_tau0.1_contrast", A.FORM_RAS, 4),
    ("lap32_box8_tau1e-12", A.FORM_RAS, 7),
    ("lap16_box4_tau50", A.FORM_ASM, 40),
    ("lap32_box8_tau1e-12", A.FORM_ASM, 40),
]


@pytest.mark.parametrize("name,form,restart", GMRES_CASES)
def test_gmres_iterations_match_oracle(name, form, restart):
    M, S, b, xo, its_o, hist, xd, st = _gmres_pair(name, form, restart)
    assert st.converged == 1
    assert abs(st.iterations - its_o) <= 1, (st.iterations, its_o)
    assert st.true_rel_residual <= 1.5e-8, st.true_rel_residual
    if st.iterations == its_o:
        # the estimate |g_{j+1}| / ||b|| at exit, against the oracle's: 1e-6
        # relative, plus 20x the oracle's relabelling envelope of one
        # application (absolute, relative to ||b||)
        bar = 1e-6 * max(hist[its_o], 1e-14) + 1e-13 + 20 * _envelope(name, form)
        assert abs(st.rel_residual - hist[its_o]) <= bar


@pytest.mark.parametrize("name,form,restart", [("lap18_box6_ov2_tau0.5", A.FORM_DEFLATED, 30),
                                               ("diff10_bfs_ov1_tau0.1_contrast", A.FORM_DEFLATED, 30),
                                               ("diff8_bfs_ov1_tau0.5", A.FORM_RAS, 6),
                                               ("lap32_box8_tau1e-12", A.FORM_ASM, 40)])
def test_gmres_solution_matches_oracle(name, form, restart):
    M, S, b, xo, its_o, hist, xd, st = _gmres_pair(name, form, restart, rtol=1e-12, maxit=600)
    x = xd.cpu().numpy()
    xs = np.linalg.solve(S.A.toarray(), b)
    assert np.linalg.norm(x - xo) <= (1e-10 + 20 * _envelope(name, form)) * np.linalg.norm(xo)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_gmres_reproducible_and_initial_guess():
    M, part, N, ov, tau, S, dA, dpart, P = _case("diff8_bfs_ov1_tau0.5")
    b = synth.rhs(M.n, 2)
    bd = to_device(b)
    x1, x2 = torch.zeros_like(bd), torch.zeros_like(bd)
    s1 = P.gmres(bd, x1, form=A.FORM_RAS, restart=5)
    s2 = P.gmres(bd, x2, form=A.FORM_RAS, restart=5)
    assert torch.equal(x1, x2) and s1.iterations == s2.iterations
    # restarting from the solution: converged at the first step
    x3 = x1.clone()
    s3 = P.gmres(bd, x3, form=A.FORM_DEFLATED, restart=30, rtol=1e-6)
    assert s3.converged == 1 and s3.iterations <= 1
    assert s3.true_rel_residual <= 1.5e-8


def test_gmres_zero_rhs_several_rhs_and_errors():
    M, part, N, ov, tau, S, dA, dpart, P = _case("lap16_box4_tau0.5")
    z = torch.zeros(M.n, dtype=torch.float64, device="cuda")
    x = torch.ones_like(z)
    st = P.gmres(z, x, form=A.FORM_DEFLATED)
    assert st.converged == 1 and st.iterations == 0 and torch.count_nonzero(x) == 0
    B = synth.rhs(M.n, 4, nrhs=3)
    Bd = to_device(B)
    X = torch.zeros_like(Bd)
    P.gmres(Bd, X, form=A.FORM_DEFLATED, nrhs=3, rtol=1e-10)
    for k in range(3):
        assert np.linalg.norm(B[k] - S.A @ X[k].cpu().numpy()) <= 1.5e-10 * np.linalg.norm(B[k])
    b = to_device(synth.rhs(M.n, 1))
    x = torch.zeros_like(b)
    for bad in (0, A.GMRES_MAX_RESTART + 1):
        with pytest.raises(A.AmddError) as e:
            P.gmres(b, x, restart=bad)
        assert e.value.status == 1
    with pytest.raises(A.AmddError) as e:
        P.gmres(b, x, form=7)
    assert e.value.status == 1
    with pytest.raises(A.AmddError) as e:
        P.apply_form(9, b, x)
    assert e.value.status == 1
    st = P.gmres(b, x, form=A.FORM_ASM, restart=10, maxit=3, allow_noconv=True)
    assert st.converged == 0 and st.iterations == 3
    with pytest.raises(A.AmddError) as e:
        P.gmres(b, torch.zeros_like(b), form=A.FORM_ASM, restart=10, maxit=3)
    assert e.value.status == 3


def test_one_level_negative_control():
    """Sec. 4.1: the one-level methods need many more GMRES iterations than
    the deflated two-level method on the same problem."""
    M, S, b, xo, its_o, hist, xd, st_def = _gmres_pair("lap32_box8_tau1e-12", A.FORM_DEFLATED, 30)
    _, _, _, _, _, _, _, st_ras = _gmres_pair("lap32_box8_tau1e-12", A.FORM_RAS, 30)
    assert st_def.converged == 1 and st_ras.converged == 1
    assert st_ras.iterations >= 3 * st_def.iterations, (st_ras.iterations, st_def.iterations)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_deflated_gmres(prec):
    """Mixed forms: FP32 local solves inside the deflated preconditioner;
    GMRES (FP64) reaches a true residual of 1e-8 within +-10% (at least +-1)
    of the oracle's iteration count at the same eps (the FP32 splitting of
    precision 1 takes eps = 2^-23, which changes the coarse space)."""
    M, part, N, ov, tau = CASES["diff8_bfs_ov1_tau0.5"]()
    S = O.setup(M, part, N, ov, tau, eps=2.0 ** -23 if prec == 1 else O.EPS)
    b = synth.rhs(M.n, 0)
    _, its_o, _ = O.gmres(S.A, b, lambda v: O.apply_deflated(S, v), restart=30, rtol=1e-8)
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    o = A.opts_default()
    o.precision = prec
    P = Preconditioner(dA, dpart, N, ov, tau, opts=o)
    try:
        bd = to_device(b)
        xd = torch.zeros_like(bd)
        st = P.gmres(bd, xd, form=A.FORM_DEFLATED, restart=30, rtol=1e-8)
        assert st.converged == 1
        assert abs(st.iterations - its_o) <= max(1, int(0.1 * its_o)), (st.iterations, its_o)
        x = xd.cpu().numpy()
        assert np.linalg.norm(b - S.A @ x) <= 1.5e-8 * np.linalg.norm(b)
    finally:
        P.close()
