"""The rounding-robust Schur complement of the splitting (Sec. 3.2,
Remark 3.2), through the C ABI.

On high-contrast elasticity the [Omega_Gi, Omega_Di] block of Abar_ii has
eigenvalues at the shift sigma_1 eps, which is the size of the rounding
error of forming Abar_ii in FP64: its Cholesky then loses definiteness on
some subdomains (and the oracle's LAPACK Cholesky fails outright on the
layer-1 problem below on some platforms).  The library detects a pivot below
0.9 x the shift and recomputes that subdomain's Schur complement as
delta (I + C_I^T (C_R C_R^T + delta I)^{-1} C_I) (push-through identity) from
a Jacobi SVD of C_R, which is positive definite by construction.

Bars: the selection p_i of every subdomain equals the oracle's at a shift
where the oracle is robust (eps = 2^-48: the selected eps-cluster has
lambda ~ 1e5-1e6, far above 1/tau = 2, so the count does not depend on
eps), and PCG reaches 1e-8 within +-1 iteration of that oracle."""
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


@pytest.mark.parametrize("layer", [1, 2])
@pytest.mark.parametrize("prec", [0, 2])
def test_elasticity_on_the_rounding_edge(layer, prec):
    M, _, xyz = synth.elasticity3d(5, layer=layer)
    part = synth.box_partition_dofs(xyz, (3, 3, 3))
    N = int(part.max()) + 1
    S = O.setup(M, part, N, 1, 0.5, eps=2.0 ** -48)
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    o = A.opts_default()
    o.precision = prec
    P = Preconditioner(dA, dpart, N, 1, 0.5, opts=o)
    try:
        info = P.info()
        assert 0 <= info.robust_schur <= N
        for i, s in enumerate(S.subs):
            assert A.get_subdomain(P.h, i)[3] == s.p, f"subdomain {i}"
            lam = A.get_eigenvalues(P.h, i)
            assert np.all(lam[np.isfinite(lam)] >= 1.0 - 1e-6)  # every non-zero eigenvalue >= 1
        b = synth.rhs(M.n, 0)
        _, its, _ = O.pcg(S.A, b, lambda v: O.apply(S, v), rtol=1e-8)
        bd = to_device(b)
        xd = torch.zeros_like(bd)
        st = P.solve(bd, xd, rtol=1e-8)
        assert st.converged == 1 and abs(st.iterations - its) <= 1, (st.iterations, its)
        assert st.true_rel_residual <= 1.5e-8
    finally:
        P.close()
