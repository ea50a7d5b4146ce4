"""Parity at the benchmark's own workload: the 3D channelled diffusion on 24^3
(16 BFS subdomains of 256..2048 cells, overlap 2, tau = 100), in the launch
configuration bench.py times (default options, mixed and plain FP64 forms).

The oracle cannot set up the whole problem in seconds (its dense coarse
Cholesky alone is of order n_C^3 = 2.6e12), so the checks use what it computes
one subdomain at a time, and a closed form that holds at this tau:
  * sampled subdomains (three, seeded): singular values of X_i, eigenvalues of
    eq. (Zi) as mu = 1/lambda and the selection p_i, against the oracle's local
    steps (Sec. 2.1 sets, eq. (Xi), Sec. 3.2 splitting, eq. (Zi)) in FP64.  The
    bars take the oracle's own FP64 envelope on the subdomain: the spread of
    its results under one seeded relabelling of the sets and, for mu, also
    under a normwise backward perturbation of X_i of size sqrt(n_i) u sigma_1.
    That is the probabilistic rounding bound of the length-n_i products by
    which the FP64 splitting rotates X_i. The Schur complement onto Omega_Ii
    amplifies such perturbations through the shifted Abar_RR (Sec. 3.2), so
    mu carries far more than u of them;
  * with tau = 100 every eigenvalue of eq. (Zi) is selected in FP64 (n_C = n),
    so R_0^T E^{-1} R_0 = A^{-1} for any basis, and one apply is
        z = A^{-1} r + sum_i R_i^T A_ii^{-1} R_i r,
    with A^{-1} r by a sparse direct solve and the local terms by dense FP64
    Cholesky solves: compared entry by entry relative to max |z|, within
    max(1e-10, 20 eta) with eta the reference's own FP64 envelope (the same
    solve with another elimination order), plain FP64 form;
  * PCG with that closed-form preconditioner in FP64 on the host gives the
    reference iteration count: the plain form within +-1, the mixed form
    within +-10% (at least +-1), both with a true residual of 1e-8.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import synth
from oracle import amdd_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, Preconditioner, to_device  # noqa: E402


@pytest.fixture(scope="module")
def headline():
    w = synth.workload_diffusion3d(m=24, N=16, lo=256, hi=2048, overlap=2, tau=100.0)
    As = O.to_scipy(w["A"])
    dA = DeviceMatrix(w["A"])
    dpart = torch.from_numpy(np.asarray(w["part"], np.int32)).cuda()
    P = {}
    for prec in (0, 1):
        o = A.opts_default()
        o.precision = prec
        P[prec] = Preconditioner(dA, dpart, w["N"], w["overlap"], w["tau"], o)
    sets = [O.subdomain_sets(As, w["part"], i, w["overlap"]) for i in range(w["N"])]
    chols = []
    for I, G, D in sets:
        om = np.concatenate([I, G])
        chols.append((om, sla.cho_factor(As[om][:, om].toarray(), lower=True)))
    lus = [spla.splu(As.tocsc()), spla.splu(As.tocsc(), permc_spec="NATURAL")]

    def apply_ref(r, which=0):
        z = lus[which].solve(r)
        for om, c in chols:
            z[om] += sla.cho_solve(c, r[om])
        return z

    yield w, As, P, sets, apply_ref
    for p in P.values():
        p.close()


def _mu(lam):
    with np.errstate(divide="ignore"):
        return np.sort(np.where(np.isinf(lam), 0.0, 1.0 / lam))


def test_headline_sampled_subdomains(headline):
    w, As, P, sets, _ = headline
    Pp = P[0]
    assert Pp.info().n_C == w["A"].n
    for i in np.random.default_rng(11).choice(w["N"], 3, replace=False):
        I, G, D = sets[i]
        nI, nG, nD, p = A.get_subdomain(Pp.h, int(i))
        assert (nI, nG, nD) == (len(I), len(G), len(D)) and p == len(I)
        Aii, X = O.local_matrices(As, I, G, D)
        Abar, sig = O.splitting_root(X, O.EPS)
        lam, _, keep = O.local_eigenproblem(Aii, Abar, len(I), w["tau"])
        assert keep.sum() == len(I)
        # the oracle's envelope: the same subdomain with its sets relabelled
        rng = np.random.default_rng(int(i) + 5)
        Ip, Gp, Dp = rng.permutation(I), rng.permutation(G), rng.permutation(D)
        Aii2, X2 = O.local_matrices(As, Ip, Gp, Dp)
        Abar2, sig2 = O.splitting_root(X2, O.EPS)
        lam2, _, _ = O.local_eigenproblem(Aii2, Abar2, len(I), w["tau"])
        so = np.sort(sig)[::-1]
        eta_s = np.abs(np.sort(sig2)[::-1] - so).max()
        sg = A.get_singular_values(Pp.h, int(i))
        assert np.all(np.abs(sg - so) <= 1e-10 * so + 20 * eta_s), f"sigma, subdomain {i}"
        mo = _mu(lam)
        eta_m = np.abs(_mu(lam2) - mo).max()
        n, nt = X.shape
        E = rng.standard_normal((n, nt)) * (np.sqrt(n) * 2.0**-53 * so[0] / (np.sqrt(n) + np.sqrt(nt)))
        Abar3, _ = O.splitting_root(X + E, O.EPS)
        lam3, _, _ = O.local_eigenproblem(Aii, Abar3, len(I), w["tau"])
        eta_m = max(eta_m, np.abs(_mu(lam3) - mo).max())
        mg = _mu(A.get_eigenvalues(Pp.h, int(i)))
        worst = np.max(np.abs(mg - mo) / (1e-8 * mo + 20 * eta_m + 1e-300))
        assert worst <= 1.0, f"mu, subdomain {i}: {worst:.2f}"


def test_headline_apply_closed_form(headline):
    w, As, P, sets, apply_ref = headline
    r = np.random.default_rng(3).uniform(-1, 1, w["A"].n)
    zo = apply_ref(r)
    # FP64 envelope of the reference itself: the sparse direct solve with
    # another elimination order (A has contrast 1e6, so A^{-1} r carries
    # rounding of order kappa(A) u)
    eta = np.abs(apply_ref(r, 1) - zo).max() / np.abs(zo).max()
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P[0].apply(rd, zd)
    err = np.abs(zd.cpu().numpy() - zo).max() / np.abs(zo).max()
    assert err <= max(1e-10, 20 * eta), (err, eta)
    P[1].apply(rd, zd)
    err = np.abs(zd.cpu().numpy() - zo).max() / np.abs(zo).max()
    assert err <= 1e-3, err  # FP32 local factors and splitting


def test_headline_pcg_iterations(headline):
    w, As, P, sets, apply_ref = headline
    b = w["b"]
    _, its_o, _ = O.pcg(As, b, apply_ref, rtol=1e-8)
    bd = to_device(b)
    for prec, slack in ((0, 1), (1, max(1, int(np.ceil(0.1 * its_o))))):
        x = torch.zeros_like(bd)
        st = P[prec].solve(bd, x, rtol=1e-8)
        assert st.converged == 1 and st.true_rel_residual <= 2e-8
        assert abs(st.iterations - its_o) <= slack, (prec, st.iterations, its_o)
        xr = x.cpu().numpy()
        assert np.linalg.norm(b - As @ xr) <= 2e-8 * np.linalg.norm(b)
