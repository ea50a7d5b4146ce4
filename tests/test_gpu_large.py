"""Parity on subdomains of 1.5k to 3k unknowns: 3D channelled diffusion with
seeded BFS subdomains and overlap 2, the shapes of the 3D configurations at a
size the oracle sets up in seconds.  At these sizes the rows of X_i (and of
[T | I] for the eigenvectors) do not fit in shared memory, so the one-sided
Jacobi solvers take their block-pair form (rows in global memory), and the
Householder reduction, the blocked Cholesky factors and the local solves run
on matrices of the 3D configurations' order.

Bars (FP64, precision = 0), per subdomain i, against the FP64 oracle:
  * singular values of X_i: |dsigma_j| <= 1e-10 sigma_j + 20 eta_sigma;
  * eigenvalues of eq. (Zi) as mu = 1/lambda: |dmu| <= 1e-8 mu + 20 eta_mu;
  * p_i exactly, n_C exactly;
  * one apply, entry by entry: |dz| <= max(1e-10, 20 eta_apply) ||z||_inf;
  * PCG iterations to 1e-8 within +-1, true residual <= 1.5e-8.
eta is the oracle's own FP64 envelope: the largest change of its result when
the unknowns are relabelled (one seeded permutation).
Mixed forms (precision 1 and 2): the selection equals the oracle's at the
form's eps; PCG reaches a true residual of 1e-8 within +-10% (at least +-1)
of the iteration count of the oracle with the same selection (the plain FP64
oracle, or for the FP32 splitting with tau < 1 the oracle at eps = 2^-23).
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


def _diff(m, N, lo, hi, tau, seed=3):
    M = synth.diffusion3d(m, sigma=2.0, corr=4.0, n_channels=4, seed=seed)
    part = synth.bfs_partition(M, N, seed, lo, hi)
    return M, part, int(part.max()) + 1, 2, tau


CASES = {
    "diff16_bfs4_ov2_tau0.5": lambda: _diff(16, 4, 512, 2048, 0.5),
    "diff16_bfs4_ov2_tau100": lambda: _diff(16, 4, 512, 2048, 100.0),
    "diff20_bfs4_ov2_tau0.5": lambda: _diff(20, 4, 1024, 4096, 0.5),
}

_cache = {}


def _mu(lam):
    with np.errstate(divide="ignore"):
        return np.sort(np.where(np.isinf(lam), 0.0, 1.0 / lam))


def _case(name):
    if name not in _cache:
        M, part, N, ov, tau = CASES[name]()
        S = O.setup(M, part, N, ov, tau)
        # the oracle's FP64 envelope under one relabelling of the unknowns
        perm = np.random.default_rng(101).permutation(M.n)
        inv = np.argsort(perm)
        Sp = O.setup(S.A[perm][:, perm].tocsr(), np.asarray(part)[perm], N, ov, tau)
        r = np.random.default_rng(7).uniform(-1, 1, M.n)
        zo = O.apply(S, r)
        zp = O.apply(Sp, r[perm])[inv]
        eta = {"apply": np.abs(zp - zo).max() / np.abs(zo).max(),
               "mu": [np.abs(_mu(t.lam) - _mu(s.lam)).max() for s, t in zip(S.subs, Sp.subs)],
               "sigma": [np.abs(np.sort(t.sigma)[::-1] - np.sort(s.sigma)[::-1]).max()
                         for s, t in zip(S.subs, Sp.subs)]}
        dA = DeviceMatrix(M)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
        P = Preconditioner(dA, dpart, N, ov, tau)
        _cache[name] = (M, part, N, ov, tau, S, eta, r, zo, dA, dpart, P)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_large_subdomains_fp64(name):
    M, part, N, ov, tau, S, eta, r, zo, dA, dpart, P = _case(name)
    assert max(len(s.omega) for s in S.subs) >= 1500
    for i, s in enumerate(S.subs):
        sg = A.get_singular_values(P.h, i)
        so = np.sort(s.sigma)[::-1]
        assert np.all(np.abs(sg - so) <= 1e-10 * so + 20 * eta["sigma"][i]), f"sigma, subdomain {i}"
        mo, mg = _mu(s.lam), _mu(A.get_eigenvalues(P.h, i))
        worst = np.max(np.abs(mg - mo) / (1e-8 * mo + 20 * eta["mu"][i]))
        assert worst <= 1.0, f"mu, subdomain {i}: {worst:.2f}"
        assert A.get_subdomain(P.h, i)[3] == s.p, f"p, subdomain {i}"
    assert P.info().n_C == S.nC
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P.apply(rd, zd)
    zg = zd.cpu().numpy()
    bar = max(1e-10, 20 * eta["apply"])
    assert np.abs(zg - zo).max() <= bar * np.abs(zo).max()
    b = synth.rhs(M.n, 0)
    _, its_o, _ = O.pcg(S.A, b, lambda v: O.apply(S, v), rtol=1e-8)
    bd = to_device(b)
    x = torch.zeros_like(bd)
    st = P.solve(bd, x, rtol=1e-8)
    assert st.converged == 1 and abs(st.iterations - its_o) <= 1 and st.true_rel_residual <= 1.5e-8


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_large_subdomains_mixed(name, prec):
    M, part, N, ov, tau, S, eta, r, zo, dA, dpart, P = _case(name)
    Sr = O.setup(M, part, N, ov, tau, eps=EPS32) if prec == 1 else S
    o = A.opts_default()
    o.precision = prec
    Q = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        for i, s in enumerate(Sr.subs):
            assert A.get_subdomain(Q.h, i)[3] == s.p, f"p, subdomain {i}"
        b = synth.rhs(M.n, 0)
        Sit = Sr if tau < 1.0 else S
        _, its_o, _ = O.pcg(Sit.A, b, lambda v: O.apply(Sit, v), rtol=1e-8)
        bd = to_device(b)
        x = torch.zeros_like(bd)
        st = Q.solve(bd, x, rtol=1e-8)
        assert st.converged == 1 and st.true_rel_residual <= 2e-8
        assert abs(st.iterations - its_o) <= max(1, int(np.ceil(0.1 * its_o))), (st.iterations, its_o)
    finally:
        Q.close()


def test_sparse_local_factors_beyond_shared_memory():
    """On subdomains of 1.5k to 2k unknowns (3D, overlap 2) a sparse factor does
    not fit in shared memory: local_solver = 1 is AMDD_ERR_INVALID and
    local_solver = 2 keeps the dense inverse factors."""
    M, part, N, ov, tau, S, eta, r, zo, dA, dpart, P = _case("diff16_bfs4_ov2_tau100")
    o = A.opts_default()
    o.local_solver = 1
    with pytest.raises(A.AmddError) as e:
        Preconditioner(dA, dpart, N, ov, tau, o)
    assert e.value.status == 1
    o.local_solver = 2
    Q = Preconditioner(dA, dpart, N, ov, tau, o)
    try:
        assert Q.info().sparse_local_nnz == 0
    finally:
        Q.close()
