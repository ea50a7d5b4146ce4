"""Failure detection of the bounded device waits without a GPU fault: the wait
that the persistent block-pair Jacobi sweep uses for its round counters runs
on a flag that is set (the call returns) and on one that nothing sets (the
kernel gives up after about 2 ms, latches the timeout and returns; the call
reports AMDD_ERR_TIMEOUT).  The context stays usable: an SpMV afterwards
equals the host product."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2109_05908_gb300 import amdd as A  # noqa: E402
from paper_2109_05908_gb300.device import DeviceMatrix, to_device  # noqa: E402


def test_bounded_wait_reports_timeout_and_the_context_survives():
    s = torch.cuda.current_stream().cuda_stream
    A.wait_selftest(True, s)
    with pytest.raises(A.AmddError) as e:
        A.wait_selftest(False, s)
    assert e.value.status == 5  # AMDD_ERR_TIMEOUT
    A.wait_selftest(True, s)
    M = synth.laplace2d(8)
    dA = DeviceMatrix(M)
    x = np.random.default_rng(0).uniform(-1, 1, M.n)
    xd = to_device(x)
    yd = torch.empty_like(xd)
    A.spmv(dA.csr, xd.data_ptr(), yd.data_ptr(), s)
    rows = np.repeat(np.arange(M.n), np.diff(M.rowptr))
    y = np.zeros(M.n)
    np.add.at(y, rows, M.val * x[M.colind])
    assert np.abs(yd.cpu().numpy() - y).max() <= 1e-14 * np.abs(y).max()
