"""The mixed-precision forms against the FP64 CPU oracle.

precision = 1: local factors, local solves, SVD, splitting and eigensolve in
FP32; E, its factor, the coarse solve and PCG in FP64.  Sec. 3.2 takes the
shift eps of the splitting as the machine precision of the arithmetic, so the
FP32 stage runs with eps = 2^-23; the reference is the oracle at that eps.

precision = 2: the splitting (SVD of X_i, Abar_ii, its Schur complement) in
FP64 with eps = 2^-52; local factors, local solves, T and its eigensolve in
FP32; E and PCG in FP64.  The reference is the plain FP64 oracle.

Bars, against the reference of each form:
  * the same selection (count per subdomain) and coarse dimension;
  * one apply within 1e-3 relative of the oracle's FP64 apply.  This is a
    structural check: FP32 local solves alone move the apply by ~1e-7
    (measured with FP32 Cholesky solves inside the oracle's apply), but FP32
    eigensolves perturb the selected spans by up to u32 ||T|| / gap, 1.3e-4
    measured on the 1e5-contrast case.  With the FP32 splitting the bar is
    max(1e-3, 4 u32 kappa_X), kappa_X the largest sigma_1 / sigma_min of the
    X_i: an FP32 SVD fixes singular directions only to u32 sigma_1 (layered
    elasticity has kappa_X ~ 4e6);
  * PCG reaches a true relative residual of 1e-8 against the FP64 matrix with
    the reference's iteration count +-10% (at least +-1), and its Lanczos
    condition estimate lies under the bound of Sec. 3.2;
  * the mixed form with the FP64 splitting (precision = 2), and the FP32 form
    whenever its selection is the plain one (tau >= 1: every eigenvalue is
    selected), take the PLAIN FP64 oracle's (eps = 2^-52) iteration count
    +-10% (at least +-1).  With tau < 1 the FP32 splitting's eps = 2^-23
    changes which eigenvalues pass the threshold (the eps-cluster moves with
    eps), so precision = 1 is a different coarse space there: measured 41
    against 28 iterations on the layered elasticity, 19 against 23 on a 3D
    diffusion with 2k-unknown subdomains;
  * bitwise reproducible.
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

EPS32 = 2.0 ** -23
EPS64 = 2.0 ** -52


def _lap(m, box, ov, tau):
    M = synth.laplace2d(m)
    part = synth.box_partition_2d(m, box)
    return M, part, int(part.max()) + 1, ov, tau, synth.rhs(M.n, 0)


def _diff(m, N, seed, ov, tau, lo, hi, cv=1e3, sigma=1.0):
    M = synth.diffusion3d(m, sigma=sigma, corr=2.0, n_channels=2, seed=seed, channel_value=cv)
    part = synth.bfs_partition(M, N, seed=seed, min_size=lo, max_size=hi)
    return M, part, int(part.max()) + 1, ov, tau, synth.rhs(M.n, 0)


def _elas(ne, box, layer, ov, tau):
    M, f, xyz = synth.elasticity3d(ne, layer=layer)
    part = synth.box_partition_dofs(xyz, (box, box, box))
    return M, part, int(part.max()) + 1, ov, tau, f


CASES = {
    "lap64_box16_tau50_C1": lambda: _lap(64, 16, 1, 50.0),
    "lap16_box4_tau0.5": lambda: _lap(16, 4, 1, 0.5),
    "diff8_bfs_ov1_tau0.5": lambda: _diff(8, 6, 1, 1, 0.5, 40, 160),
    "diff9_bfs_ov2_tau100": lambda: _diff(9, 5, 2, 2, 100.0, 60, 220),
    "diff10_bfs_ov1_tau0.1_contrast": lambda: _diff(10, 8, 4, 1, 0.1, 60, 200, cv=1e5, sigma=1.5),
    "elas6_layer2_ov1_tau0.5": lambda: _elas(6, 4, 2, 1, 0.5),
    "elas5_layer2_ov2_tau100": lambda: _elas(5, 3, 2, 2, 100.0),
}
PARAMS = [(p, c) for p in (1, 2) for c in CASES]
IDS = [f"p{p}-{c}" for p, c in PARAMS]


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, mk in CASES.items():
        M, part, N, ov, tau, b = mk()
        S = {EPS64: O.setup(M, part, N, ov, tau, eps=EPS64), EPS32: O.setup(M, part, N, ov, tau, eps=EPS32)}
        dA = DeviceMatrix(M)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        P = {}
        for prec in (1, 2):
            o = A.opts_default()
            o.precision = prec
            P[prec] = Preconditioner(dA, dpart, N, ov, tau, o)
        out[name] = (M, b, S, P)
    yield out
    for _, _, _, P in out.values():
        for p in P.values():
            p.close()


def _ref(S, prec):
    return S[EPS32] if prec == 1 else S[EPS64]


@pytest.mark.parametrize("prec,name", PARAMS, ids=IDS)
def test_mixed_selection_and_apply(built, prec, name):
    M, b, S, P = built[name]
    Sr, Pp = _ref(S, prec), P[prec]
    info = Pp.info()
    assert info.precision == prec and info.eps == (EPS32 if prec == 1 else EPS64)
    for i, s in enumerate(Sr.subs):
        assert A.get_subdomain(Pp.h, i)[3] == s.p, f"subdomain {i}"
    assert info.n_C == Sr.nC
    r = synth.rhs(M.n, 9)
    zo = O.apply(Sr, r)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    Pp.apply(rd, zd)
    bar = 1e-3
    if prec == 1:
        kx = max(s.sigma.max() / s.sigma.min() for s in Sr.subs)
        bar = max(bar, 4 * 2.0 ** -24 * kx)
    zg = zd.cpu().numpy()
    assert np.linalg.norm(zg - zo) <= bar * np.linalg.norm(zo)
    assert np.abs(zg - zo).max() <= bar * np.abs(zo).max()  # entry by entry
    z2 = torch.empty_like(rd)
    Pp.apply(rd, z2)
    assert torch.equal(zd, z2)


@pytest.mark.parametrize("prec,name", PARAMS, ids=IDS)
def test_mixed_pcg_reaches_1e8(built, prec, name):
    M, b, S, P = built[name]
    Sr, Pp = _ref(S, prec), P[prec]
    _, its_o, _ = O.pcg(Sr.A, b, lambda v: O.apply(Sr, v), rtol=1e-8)
    bd = to_device(b)
    x = torch.zeros_like(bd)
    st = Pp.solve(bd, x, rtol=1e-8)
    assert st.converged == 1
    assert st.true_rel_residual <= 2e-8
    assert abs(st.iterations - its_o) <= max(1, int(np.ceil(0.1 * its_o))), (st.iterations, its_o)
    xr = x.cpu().numpy()
    res = np.linalg.norm(b - Sr.A @ xr) / np.linalg.norm(b)
    assert res <= 2e-8
    if M.n <= 1000:
        bound = O.condition_bound(O.colouring_number(Sr), O.splitting_constant(Sr), Sr.tau)
        assert st.cond_est <= bound


@pytest.mark.parametrize("prec,name", PARAMS, ids=IDS)
def test_mixed_iterations_match_plain_oracle(built, prec, name):
    """The headline bar: the mixed forms reach 1e-8 within +-10% (at least +-1)
    of the iteration count of the plain FP64 oracle at eps = 2^-52 (the FP32
    splitting only where its selection is the plain one, tau >= 1)."""
    M, b, S, P = built[name]
    if prec == 1 and S[EPS64].tau < 1.0:
        pytest.skip("FP32 splitting with tau < 1: a different eps-cluster, compared with its own oracle")
    S64 = S[EPS64]
    _, its_o, _ = O.pcg(S64.A, b, lambda v: O.apply(S64, v), rtol=1e-8)
    bd = to_device(b)
    x = torch.zeros_like(bd)
    st = P[prec].solve(bd, x, rtol=1e-8)
    assert st.converged == 1 and st.true_rel_residual <= 2e-8
    assert abs(st.iterations - its_o) <= max(1, int(np.ceil(0.1 * its_o))), (st.iterations, its_o)


def test_mixed_batched_rhs(built):
    """Eight right-hand sides solved together in the mixed form: each reaches a
    true relative residual of 1e-8 against the FP64 matrix."""
    M, b, S, P = built["lap64_box16_tau50_C1"]
    B = synth.rhs(M.n, 31, nrhs=8)
    bd = to_device(B)
    x = torch.zeros_like(bd)
    st = P[1].solve(bd, x, nrhs=8, rtol=1e-8)
    assert st.converged == 1
    X = x.cpu().numpy()
    for k in range(8):
        assert np.linalg.norm(B[k] - S[EPS64].A @ X[k]) <= 2e-8 * np.linalg.norm(B[k])
