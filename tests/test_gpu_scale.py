"""Parity at the size `bench.py` times its bandwidth problem: the 2D Laplacian
1024 x 1024 (n = 1,048,576), 4096 boxes of 16 x 16, overlap 1, mixed form,
tau = 1e-12 (no eigenvalue above 1e12 in the FP32 splitting, so n_C = 0 and
the apply is the one-level sum of Sec. 2.1).  The oracle cannot set up all
4096 subdomains in seconds, so the checks use outputs it computes one by one
and properties that hold at any size:
  * sampled outputs: for 24 sampled unknowns g, z[g] = sum over the
    subdomains i whose Omega_i holds g of (A_ii^{-1} R_i r)[g], each local
    solve a dense FP64 Cholesky solve of the oracle's A_ii; 2e-5 relative to
    max |z| (FP32 local factors and solves);
  * symmetry of M: |u^T M v - v^T M u| <= 1e-5 |u^T M v|;
  * PCG reaches a true relative residual of 1e-8;
  * bitwise reproducibility of the apply.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import amdd_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, Preconditioner, to_device  # noqa: E402

M_SIDE, BOX = 1024, 16


@pytest.fixture(scope="module")
def big():
    M = synth.laplace2d(M_SIDE)
    part = synth.box_partition_2d(M_SIDE, BOX)
    N = int(part.max()) + 1
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(part).cuda()
    o = A.opts_default()
    o.precision = 1
    P = Preconditioner(dA, dpart, N, 1, 1e-12, opts=o)
    yield M, part, N, P
    P.close()


def test_one_level_apply_sampled(big):
    M, part, N, P = big
    assert P.info().n_C == 0
    As = O.to_scipy(M)
    r = np.random.default_rng(3).uniform(-1, 1, M.n)
    rd = to_device(r)
    zd = torch.empty_like(rd)
    P.apply(rd, zd)
    z = zd.cpu().numpy()
    rng = np.random.default_rng(4)
    samples = rng.choice(M.n, 24, replace=False)
    zmax = np.abs(z).max()
    nb = M_SIDE // BOX
    for g in samples:
        gy, gx = divmod(int(g), M_SIDE)
        # subdomains whose Omega_i (box plus one layer) holds g
        owners = set()
        for by in range(max(0, (gy - 1) // BOX), min(nb, (gy + 1) // BOX + 1)):
            for bx in range(max(0, (gx - 1) // BOX), min(nb, (gx + 1) // BOX + 1)):
                owners.add(by * nb + bx)
        ref = 0.0
        for i in owners:
            I, G, D = O.subdomain_sets(As, part, i, 1)
            om = np.concatenate([I, G])
            pos = np.flatnonzero(om == g)
            if len(pos) == 0:
                continue
            Aii, _ = O.local_matrices(As, I, G, D)
            y = sla.cho_solve(sla.cho_factor(Aii, lower=True), r[om])
            ref += y[pos[0]]
        assert abs(z[g] - ref) <= 2e-5 * zmax, (int(g), z[g], ref)


def test_symmetry_reproducibility_and_pcg(big):
    M, part, N, P = big
    rng = np.random.default_rng(5)
    u, v = rng.uniform(-1, 1, M.n), rng.uniform(-1, 1, M.n)
    ud, vd = to_device(u), to_device(v)
    mu, mv = torch.empty_like(ud), torch.empty_like(vd)
    P.apply(ud, mu)
    P.apply(vd, mv)
    a, b = float(torch.dot(vd, mu)), float(torch.dot(ud, mv))
    assert abs(a - b) <= 1e-5 * abs(a)
    mu2 = torch.empty_like(ud)
    P.apply(ud, mu2)
    assert torch.equal(mu, mu2)
    bvec = to_device(synth.rhs(M.n, 0))
    x = torch.zeros_like(bvec)
    st = P.solve(bvec, x, rtol=1e-8, maxit=2000)
    assert st.converged == 1 and st.true_rel_residual <= 1.5e-8
