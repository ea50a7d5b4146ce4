"""The allocation-free true-residual entry point (for callers that cannot
allocate device memory) gives bit for bit the residual amdd_pcg_solve reports
for the same solution (same SpMV lane width, same fixed reduction order), on
two calls in a row (its static scratch is reused and must be re-initialised by
every call); it agrees with ||b - A x|| and ||b|| computed on the host for a
non-zero x, and rejects sizes beyond its static scratch.  Collected last so
that a run stopping at the first failure has run every other test first; it
also passes alone in a fresh process."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, Preconditioner, to_device  # noqa: E402


def test_matches_pcg_true_residual_twice():
    w = synth.workload_c1()
    dA = DeviceMatrix(w["A"])
    part = torch.from_numpy(np.asarray(w["part"], np.int32)).cuda()
    P = Preconditioner(dA, part, w["N"], w["overlap"], w["tau"])
    try:
        b = to_device(w["b"])
        x = torch.zeros_like(b)
        st = P.solve(b, x, rtol=1e-8)
        stream = torch.cuda.current_stream().cuda_stream
        r1 = A.true_residual_noalloc(dA.csr, b.data_ptr(), x.data_ptr(), stream)
        r2 = A.true_residual_noalloc(dA.csr, b.data_ptr(), x.data_ptr(), stream)
        assert r1 == r2
        assert r1[1] == pytest.approx(float(np.linalg.norm(w["b"])), rel=1e-14)
        # the same kernels in the same order: the same bits
        assert r1[0] / r1[1] == st.true_rel_residual
        # independent host check at a non-zero x (the PCG solution itself)
        xs = x.cpu().numpy()
        M = w["A"]
        rows = np.repeat(np.arange(M.n), np.diff(M.rowptr))
        ax = np.zeros(M.n)
        np.add.at(ax, rows, M.val * xs[M.colind])
        res_host = float(np.linalg.norm(w["b"] - ax))
        assert r1[0] == pytest.approx(res_host, rel=1e-6, abs=1e-15 * float(np.linalg.norm(w["b"])))
        # a rougher non-zero x: the residual is O(||b||), so the relative bar is tight
        rng = np.random.Generator(np.random.PCG64(7))
        xr = rng.uniform(-1.0, 1.0, M.n)
        axr = np.zeros(M.n)
        np.add.at(axr, rows, M.val * xr[M.colind])
        xr_d = to_device(xr)
        r4 = A.true_residual_noalloc(dA.csr, b.data_ptr(), xr_d.data_ptr(), stream)
        assert r4[0] == pytest.approx(float(np.linalg.norm(w["b"] - axr)), rel=1e-12)
        # a different x between calls: the scratch holds the last call's values
        x2 = torch.zeros_like(b)
        r3 = A.true_residual_noalloc(dA.csr, b.data_ptr(), x2.data_ptr(), stream)
        assert r3[0] == pytest.approx(r3[1], rel=1e-14)  # x = 0: residual is b
    finally:
        P.close()


def test_rejects_sizes_beyond_the_static_scratch():
    M = synth.laplace2d(8)
    dA = DeviceMatrix(M)
    big = A.make_csr(A.NOALLOC_MAX_N + 1, dA.nnz, dA.rowptr.data_ptr(), dA.colind.data_ptr(), dA.val.data_ptr())
    x = torch.zeros(M.n, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AmddError) as e:
        A.true_residual_noalloc(big, x.data_ptr(), x.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
