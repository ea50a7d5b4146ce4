"""The mixed-precision form (local factors, local solves, SVD, splitting and
eigensolve in FP32; E, its factor, the coarse solve and PCG in FP64) against
the FP64 CPU oracle.  Sec. 3.2 takes the shift eps of the splitting as the
machine precision of the arithmetic, so the FP32 stage runs with eps = 2^-23
and is compared with the oracle at that eps.  Bars:
  * the same selection (count per subdomain) and coarse dimension;
  * one apply within 1e-3 relative of the oracle's FP64 apply.  This is a
    structural check: FP32 local solves alone move the apply by ~1e-7
    (measured with FP32 Cholesky solves inside the oracle's apply), but FP32
    eigensolves perturb the selected spans by up to u32 ||T|| / gap, 1.3e-4
    measured on the 1e5-contrast case;
  * PCG reaches a true relative residual of 1e-8 against the FP64 matrix with
    the iteration count of the plain FP64 oracle (eps = 2^-52) +-10% (at
    least +-1), and its Lanczos condition estimate lies under the bound of
    Sec. 3.2;
  * bitwise reproducible."""
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
    "lap64_box16_tau50_C1": lambda: _lap(64, 16, 1, 50.0),
    "lap16_box4_tau0.5": lambda: _lap(16, 4, 1, 0.5),
    "diff8_bfs_ov1_tau0.5": lambda: _diff(8, 6, 1, 1, 0.5, 40, 160),
    "diff9_bfs_ov2_tau100": lambda: _diff(9, 5, 2, 2, 100.0, 60, 220),
    "diff10_bfs_ov1_tau0.1_contrast": lambda: _diff(10, 8, 4, 1, 0.1, 60, 200, cv=1e5, sigma=1.5),
}


EPS32 = 2.0 ** -23


@pytest.fixture(scope="module")
def built():
    out = {}
    for name, mk in CASES.items():
        M, part, N, ov, tau = mk()
        S = O.setup(M, part, N, ov, tau, eps=EPS32)
        S64 = O.setup(M, part, N, ov, tau)
        o = A.opts_default()
        o.precision = 1
        P = Preconditioner(DeviceMatrix(M), torch.from_numpy(np.asarray(part, np.int32)).cuda(), N, ov, tau, o)
        out[name] = (M, S, S64, P)
    yield out
    for _, _, _, P in out.values():
        P.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_selection_and_apply(built, name):
    M, S, S64, P = built[name]
    assert P.info().precision == 1 and P.info().eps == EPS32
    for i, s in enumerate(S.subs):
        assert A.get_subdomain(P.h, i)[3] == s.p
    assert P.info().n_C == S.nC
    r = synth.rhs(M.n, 9)
    zo = O.apply(S, r)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P.apply(rd, zd)
    assert np.linalg.norm(zd.cpu().numpy() - zo) <= 1e-3 * np.linalg.norm(zo)
    z2 = torch.empty_like(rd)
    P.apply(rd, z2)
    assert torch.equal(zd, z2)


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_pcg_reaches_1e8(built, name):
    M, S, S64, P = built[name]
    b = synth.rhs(M.n, 0)
    _, its_o, _ = O.pcg(S64.A, b, lambda v: O.apply(S64, v), rtol=1e-8)
    bd = to_device(b)
    x = torch.zeros_like(bd)
    st = P.solve(bd, x, rtol=1e-8)
    assert st.converged == 1
    assert st.true_rel_residual <= 2e-8
    assert abs(st.iterations - its_o) <= max(1, int(np.ceil(0.1 * its_o)))
    xr = x.cpu().numpy()
    res = np.linalg.norm(b - S.A @ xr) / np.linalg.norm(b)
    assert res <= 2e-8
    if M.n <= 1000:
        bound = O.condition_bound(O.colouring_number(S), O.splitting_constant(S), S.tau)
        assert st.cond_est <= bound
