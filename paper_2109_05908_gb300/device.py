"""Device-side marshalling for the C ABI: host CSR / partitions / vectors as
CUDA tensors owned by torch (memory and streams only), and the matching
`amdd_csr` descriptor."""
from __future__ import annotations

import numpy as np
import torch

from . import amdd as _a


class DeviceMatrix:
    """A CSR matrix (n, rowptr int64, colind int32, val float64) copied to a
    CUDA device; `.csr` is the amdd_csr descriptor that points at it."""

    def __init__(self, A, device="cuda"):
        self.n = int(A.n)
        self.nnz = int(A.rowptr[-1])
        self.rowptr = torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int64)).to(device)
        self.colind = torch.from_numpy(np.ascontiguousarray(A.colind, dtype=np.int32)).to(device)
        self.val = torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(device)
        self.csr = _a.make_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.colind.data_ptr(),
                               self.val.data_ptr())


def to_device(x, dtype=None, device="cuda") -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def stream_ptr() -> int:
    """The current torch CUDA stream as a raw cudaStream_t value."""
    return torch.cuda.current_stream().cuda_stream


class Preconditioner:
    """Owns an amdd handle built on a DeviceMatrix and a device partition."""

    def __init__(self, dA: DeviceMatrix, part: torch.Tensor, N: int, overlap: int, tau: float,
                 opts=None, stream: int | None = None):
        self.dA = dA
        self.part = part
        self.stream = stream_ptr() if stream is None else stream
        self.h = _a.setup(dA.csr, part.data_ptr(), N, overlap, tau, opts, self.stream)

    def apply(self, r: torch.Tensor, z: torch.Tensor, nrhs: int = 1):
        _a.apply(self.h, r.data_ptr(), z.data_ptr(), nrhs)

    def solve(self, b: torch.Tensor, x: torch.Tensor, nrhs: int = 1, rtol: float = 1e-8, maxit: int = 1000,
              allow_noconv: bool = False):
        return _a.pcg_solve(self.h, b.data_ptr(), x.data_ptr(), nrhs, rtol, maxit, allow_noconv)

    def apply_form(self, form: int, r: torch.Tensor, z: torch.Tensor, nrhs: int = 1):
        _a.apply_form(self.h, form, r.data_ptr(), z.data_ptr(), nrhs)

    def gmres(self, b: torch.Tensor, x: torch.Tensor, form: int = _a.FORM_DEFLATED, nrhs: int = 1, restart: int = 30,
              rtol: float = 1e-8, maxit: int = 1000, allow_noconv: bool = False):
        return _a.gmres_solve(self.h, form, b.data_ptr(), x.data_ptr(), nrhs, restart, rtol, maxit, allow_noconv)

    def info(self):
        return _a.get_info(self.h)

    def close(self):
        if self.h:
            _a.destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
