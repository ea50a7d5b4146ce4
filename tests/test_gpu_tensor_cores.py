"""The tcgen05 tensor-core GEMM (TF32 units, 3xTF32 split, FP32 accumulation)
through amdd_gemm_f32, against an FP64 product of the same FP32 inputs:
  * every entry within 8 k u32 max|A| max|B| (the error bound of an FP32
    multiply-add loop of length k, u32 = 2^-24), and within 4x the CUDA-core
    FMA kernel's own worst error on the same problem;
  * shapes that span several 128 x 128 tiles with ragged tails in m, n and k,
    both storage orders of A and B, alpha and beta, k = 0.
And the mixed-form setup with tensor_cores = 1: the selection of the oracle at
its eps and the PCG iteration count of the CUDA-core run.
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

U32 = 2.0 ** -24


def _gemm(m, n, k, ta, tb, alpha, beta, tc, seed):
    g = torch.Generator().manual_seed(seed)
    Ah = torch.randn((k, m) if ta else (m, k), generator=g, dtype=torch.float32)
    Bh = torch.randn((n, k) if tb else (k, n), generator=g, dtype=torch.float32)
    Ch = torch.randn((m, n), generator=g, dtype=torch.float32)
    Ad, Bd, Cd = Ah.cuda(), Bh.cuda(), Ch.cuda()
    A.gemm_f32(m, n, k, alpha, Ad.data_ptr(), Ad.shape[1], ta, Bd.data_ptr(), Bd.shape[1], tb, beta,
               Cd.data_ptr(), n, tc, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    opA = (Ah.T if ta else Ah).double()
    opB = (Bh.T if tb else Bh).double()
    ref = alpha * (opA @ opB) + beta * Ch.double()
    amax = float(Ah.abs().max()) if Ah.numel() else 0.0
    bmax = float(Bh.abs().max()) if Bh.numel() else 0.0
    bound = 8 * max(k, 1) * U32 * amax * bmax * abs(alpha) + 4 * U32 * abs(beta) * float(Ch.abs().max())
    return (Cd.cpu().double() - ref).abs().max().item(), bound


@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (300, 257, 1000), (129, 384, 37), (64, 40, 2048), (517, 131, 3)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_tensor_core_gemm_accuracy(m, n, k, ta, tb):
    err_tc, bound = _gemm(m, n, k, ta, tb, 1.0, 0.0, 1, 1)
    err_ff, _ = _gemm(m, n, k, ta, tb, 1.0, 0.0, 0, 1)
    assert err_tc <= bound, (err_tc, bound)
    assert err_tc <= 4 * err_ff + 1e-30, (err_tc, err_ff)


def test_tensor_core_gemm_alpha_beta_and_empty_k():
    err, bound = _gemm(200, 150, 300, 0, 1, -0.5, 2.0, 1, 3)
    assert err <= bound
    err, bound = _gemm(130, 140, 0, 0, 0, 1.0, 0.5, 1, 4)  # k = 0: C = beta C
    assert err <= bound


def _diff(m, N, lo, hi, tau, seed=3):
    M = synth.diffusion3d(m, sigma=2.0, corr=4.0, n_channels=4, seed=seed)
    part = synth.bfs_partition(M, N, seed, lo, hi)
    return M, part, int(part.max()) + 1, 2, tau


@pytest.mark.parametrize("case", [(16, 4, 512, 2048, 0.5), (16, 4, 512, 2048, 100.0)])
def test_mixed_setup_on_tensor_cores(case):
    M, part, N, ov, tau = _diff(*case)
    Sr = O.setup(M, part, N, ov, tau, eps=2.0 ** -23)
    dA = DeviceMatrix(M)
    dpart = torch.from_numpy(np.asarray(part, np.int32)).cuda()
    res = {}
    for tc in (0, 1):
        o = A.opts_default()
        o.precision = 1
        o.tensor_cores = tc
        o.profile = 1
        P = Preconditioner(dA, dpart, N, ov, tau, o)
        try:
            for i, s in enumerate(Sr.subs):
                assert A.get_subdomain(P.h, i)[3] == s.p, f"tc={tc}, subdomain {i}"
            b = to_device(synth.rhs(M.n, 0))
            x = torch.zeros_like(b)
            st = P.solve(b, x, rtol=1e-8)
            assert st.converged == 1 and st.true_rel_residual <= 2e-8
            prof = {p["name"]: p for p in A.get_profile(P.h)}
            res[tc] = (st.iterations, prof.get("gemm_tc_f32", {}).get("launches", 0))
        finally:
            P.close()
    assert res[1][1] > 0 and res[0][1] == 0, res  # the tensor-core kernel ran, and only when asked
    assert abs(res[1][0] - res[0][0]) <= 1, res
