"""The matrix-free local eigensolve (Sec. 3.2, eq. (invAii);
amdd_opts.eig_solver = 3) through the C ABI, against the FP64 oracle of the
same form (oracle/matrix_free.py: K = L_A^T (Abar^{-1})_II L_A formed densely,
all eigenpairs by LAPACK).

eps = 2^-23 (a shift far above FP64 rounding, see the oracle's pins).  Bars:
  * p_i equals the oracle's selection on every subdomain;
  * every computed lambda agrees with the oracle's as mu = 1/lambda to
    1e-7 relative plus 1e-6 eps (the operator's cancellation floor), the
    computed ones lead and include one at or below 1/tau unless all were
    computed; the rest are NaN;
  * the selected spans agree: A_II-orthogonal projectors within 1e-5 / gap
    (gap = relative distance of the first unselected mu to the last
    selected one);
  * PCG to 1e-8 takes the oracle's iteration count +-1 (oracle: the
    Schur-complement form at the same eps) and the dense path's +-1;
  * option errors: precision != 0, eps < 2^-30, eig_solver > 3."""
import numpy as np
import pytest

import synth
from oracle import amdd_oracle as O
from oracle import matrix_free as MF

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(240, method="thread")]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, Preconditioner, to_device  # noqa: E402

EPS = 2.0 ** -23


def _diff():
    M = synth.diffusion3d(10, sigma=1.0, corr=2.0, n_channels=2, seed=2, channel_value=1e3)
    part = synth.bfs_partition(M, 10, seed=2, min_size=50, max_size=180)
    return M, part, int(part.max()) + 1, 1, 0.5


CASES = {
    "lap24_box6_tau0.5": lambda: (synth.laplace2d(24), synth.box_partition_2d(24, 6), 16, 1, 0.5),
    "lap32_box8_ov2_tau0.7": lambda: (synth.laplace2d(32), synth.box_partition_2d(32, 8), 16, 2, 0.7),
    "diff10_bfs_tau0.5": _diff,
    "lap64_box16_tau0.5": lambda: (synth.laplace2d(64), synth.box_partition_2d(64, 16), 16, 1, 0.5),
}

_cache = {}


def _opts(solver):
    o = A.opts_default()
    o.eps = EPS
    o.eig_solver = solver
    return o


def _case(name):
    if name not in _cache:
        M, part, N, ov, tau = CASES[name]()
        ref = MF.selection(M, part, N, ov, tau, EPS)
        dA = DeviceMatrix(M)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        P = Preconditioner(dA, dpart, N, ov, tau, opts=_opts(A.EIG_MATRIX_FREE))
        _cache[name] = (M, part, N, ov, tau, ref, dA, dpart, P)
    return _cache[name]


def _mu(lam):
    return 1.0 / lam


@pytest.mark.parametrize("name", list(CASES))
def test_selection_and_eigenvalues(name):
    M, part, N, ov, tau, ref, dA, dpart, P = _case(name)
    info = P.info()
    assert info.n_C == sum(r[2] for r in ref)
    assert info.lobpcg_subdomains == N
    for i, (lam_o, _, p_o) in enumerate(ref):
        nI, _, _, p = A.get_subdomain(P.h, i)
        assert p == p_o, f"subdomain {i}: {p} vs {p_o}"
        lam = A.get_eigenvalues(P.h, i)
        c = int(np.isfinite(lam).sum())
        assert c >= p and np.all(np.isnan(lam[c:])), f"subdomain {i}"
        assert c == nI or lam[c - 1] <= 1.0 / tau, f"subdomain {i}"
        mg, mo = _mu(lam[:c]), _mu(lam_o[:c])
        assert np.all(np.abs(mg - mo) <= 1e-7 * mo + 1e-6 * EPS), f"subdomain {i}: {np.max(np.abs(mg - mo) / mo)}"


@pytest.mark.parametrize("name", list(CASES))
def test_selected_span(name):
    M, part, N, ov, tau, ref, dA, dpart, P = _case(name)
    As = O.to_scipy(M)
    checked = 0
    for i, (lam_o, U_o, p_o) in enumerate(ref):
        nI = U_o.shape[0]
        if not 0 < p_o < nI:
            continue
        I, G, D = O.subdomain_sets(As, np.asarray(part), i, ov)
        AII = As[I][:, I].toarray()
        Z = A.get_coarse_block(P.h, i)  # p x nI, A_II-orthonormal rows
        assert np.allclose(Z @ AII @ Z.T, np.eye(p_o), atol=1e-8), f"subdomain {i}"
        Pg = Z.T @ Z @ AII
        Po = U_o @ U_o.T @ AII
        mu = 1.0 / lam_o
        gap = abs(mu[p_o] - mu[p_o - 1]) / mu[p_o]
        assert np.linalg.norm(Pg - Po) <= 1e-5 / max(gap, 1e-3), f"subdomain {i}"
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_iterations(name):
    M, part, N, ov, tau, ref, dA, dpart, P = _case(name)
    S = O.setup(M, part, N, ov, tau, eps=EPS)
    b = synth.rhs(M.n, 0)
    _, its_o, _ = O.pcg(S.A, b, lambda v: O.apply(S, v), rtol=1e-8)
    bd = to_device(b)
    x = torch.zeros_like(bd)
    st = P.solve(bd, x, rtol=1e-8)
    assert st.converged == 1 and abs(st.iterations - its_o) <= 1, (st.iterations, its_o)
    assert st.true_rel_residual <= 1.5e-8
    Q = Preconditioner(dA, dpart, N, ov, tau, opts=_opts(A.EIG_DENSE))
    try:
        assert Q.info().n_C == P.info().n_C
        x2 = torch.zeros_like(bd)
        st2 = Q.solve(bd, x2, rtol=1e-8)
        assert abs(st.iterations - st2.iterations) <= 1
    finally:
        Q.close()


def test_option_errors():
    M, part, N, ov, tau = CASES["lap24_box6_tau0.5"]()
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    sp = torch.cuda.current_stream().cuda_stream
    for prec, eps, solver in ((1, EPS, 3), (2, EPS, 3), (0, 2.0 ** -52, 3), (0, 2.0 ** -31, 3), (0, EPS, 4)):
        o = _opts(solver)
        o.precision = prec
        o.eps = eps
        with pytest.raises(A.AmddError) as e:
            A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, o, sp)
        assert e.value.status == 1
    o = _opts(3)
    o.eps = 2.0 ** -30  # the smallest shift accepted
    h = A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, o, sp)
    A.destroy(h)
