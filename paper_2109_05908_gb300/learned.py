"""The learned warm start of the local eigensolve: data collection, training
and use, driving the library's kernels through the C ABI (argument
marshalling only; the features, targets, forward and backward passes and the
Adam update all run in libamdd).

A model maps the 32 features of a partially selected subdomain to a
predicted 16 x 16 projector onto its selected eigenvectors, expressed on the
orthonormal Krylov basis K_16(A_II, 1).  amdd_setup with eig_solver = 2 turns
the prediction into the first rows of the LOBPCG block; every result is still
checked (residuals, Ritz values against the bisection eigenvalues) and falls
back to the dense path when it fails.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import amdd as A
from .device import DeviceMatrix, stream_ptr

NP = A.MLP_NPARAM
NF, NB, NH = A.PROP_NF, A.PROP_NB, 256


def collect(problems, precision: int = 0, device="cuda"):
    """Features and target projectors of every partially selected subdomain of
    `problems`, an iterable of (CSR matrix, partition, N, overlap, tau).
    Returns (features (m x 32), targets (m x 16 x 16)) as float32 numpy."""
    feats, tgts = [], []
    for M, part, N, ov, tau in problems:
        dA = DeviceMatrix(M, device=device)
        dpart = torch.from_numpy(np.asarray(part, np.int32)).to(device)
        o = A.opts_default()
        o.precision = precision
        o.keep_proposal_data = 1
        h = A.setup(dA.csr, dpart.data_ptr(), N, ov, tau, o, stream_ptr())
        try:
            f, t, _ = A.proposal_export(h)
        finally:
            A.destroy(h)
        feats.append(f)
        tgts.append(t)
    return np.concatenate(feats), np.concatenate(tgts)


def init_weights(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)) and zero biases, in the
    library's parameter layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal(NF * NH) * np.sqrt(2.0 / NF), np.zeros(NH),
             rng.standard_normal(NH * NH) * np.sqrt(2.0 / NH), np.zeros(NH),
             rng.standard_normal(NH * NH) * np.sqrt(2.0 / NH), np.zeros(NH)]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == NP
    return w


class ProposalModel:
    """Weights (FP32 master and bfloat16-rounded copy), Adam moments and the
    feature standardisation, all on the device."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.device = device
        self.w = torch.from_numpy(init_weights(seed)).to(device)
        self.wb = torch.empty_like(self.w)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.t = 0
        self.mean = torch.zeros(NF, dtype=torch.float32, device=device)
        self.sd = torch.ones(NF, dtype=torch.float32, device=device)
        A.mlp_round_bf16(self.w.data_ptr(), self.wb.data_ptr(), NP, stream_ptr())
        self._prop = None

    def set_normalisation(self, feats: np.ndarray):
        """Feature means and standard deviations, computed by the library's kernel."""
        f = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).to(self.device)
        self.mean = torch.empty(NF, dtype=torch.float32, device=self.device)
        self.sd = torch.empty(NF, dtype=torch.float32, device=self.device)
        A.mlp_feature_stats(f.data_ptr(), f.shape[0], self.mean.data_ptr(), self.sd.data_ptr(), stream_ptr())

    def _inputs(self, feats: np.ndarray) -> torch.Tensor:
        f = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).to(self.device)
        x = torch.empty_like(f)
        A.mlp_normalize(f.data_ptr(), self.mean.data_ptr(), self.sd.data_ptr(), f.shape[0], x.data_ptr(),
                        stream_ptr())
        return x

    def fit(self, feats: np.ndarray, targets: np.ndarray, steps: int = 400, lr: float = 1e-3):
        """Full-batch Adam on the mean squared Frobenius error; returns the
        loss history (host floats)."""
        self.set_normalisation(feats)
        x = self._inputs(feats)
        qt = torch.from_numpy(np.ascontiguousarray(targets, np.float32).reshape(len(targets), -1)).to(self.device)
        n = x.shape[0]
        _, nwork = A.mlp_sizes(n)
        work = torch.empty(nwork, dtype=torch.float32, device=self.device)
        grad = torch.empty(NP, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        hist = []
        for _ in range(steps):
            self.t += 1
            A.mlp_train_step(self.w.data_ptr(), self.wb.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.t, lr,
                             x.data_ptr(), qt.data_ptr(), n, grad.data_ptr(), work.data_ptr(), loss.data_ptr(),
                             stream_ptr())
            hist.append(float(loss.item()))
        return hist

    def predict(self, feats: np.ndarray) -> np.ndarray:
        x = self._inputs(feats)
        n = x.shape[0]
        _, nwork = A.mlp_sizes(n)
        work = torch.empty(nwork, dtype=torch.float32, device=self.device)
        q = torch.empty((n, NB * NB), dtype=torch.float32, device=self.device)
        A.mlp_forward(self.wb.data_ptr(), x.data_ptr(), n, q.data_ptr(), work.data_ptr(), stream_ptr())
        return q.cpu().numpy().reshape(n, NB, NB)

    def proposal(self) -> A.amdd_proposal:
        """The amdd_proposal of this model (valid while the model lives)."""
        self._prop = A.amdd_proposal(self.wb.data_ptr(), self.mean.data_ptr(), self.sd.data_ptr())
        return self._prop

    def opts(self, precision: int = 0) -> A.amdd_opts:
        o = A.opts_default()
        o.precision = precision
        o.eig_solver = 2
        o.proposal = C.pointer(self.proposal())
        return o

    def save(self, path: str):
        np.savez(path, w=self.w.cpu().numpy(), mean=self.mean.cpu().numpy(), sd=self.sd.cpu().numpy())

    @classmethod
    def load(cls, path: str, device="cuda") -> "ProposalModel":
        z = np.load(path)
        mdl = cls(device=device)
        mdl.w = torch.from_numpy(z["w"]).to(device)
        mdl.wb = torch.empty_like(mdl.w)
        A.mlp_round_bf16(mdl.w.data_ptr(), mdl.wb.data_ptr(), NP, stream_ptr())
        mdl.mean = torch.from_numpy(z["mean"]).to(device)
        mdl.sd = torch.from_numpy(z["sd"]).to(device)
        return mdl
