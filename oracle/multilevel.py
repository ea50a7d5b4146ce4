"""Plain FP64 CPU oracle of the multilevel form of the preconditioner
(Sec. 3.2, last paragraph, and Sec. 4.2): the same fully algebraic
construction applied to the coarse matrix E = R_0 A R_0^T, so that the coarse
solve C_00^{-1} of the deflated method (Sec. 4.1) becomes an inexact solve:
right-preconditioned GMRES(30) to a relative tolerance of 1e-4 on E with the
two-level deflated method built on E, inside an outer flexible GMRES(30)
(Sec. 4.2).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library.

Readings where the paper is silent (each listed in the design notes):
  * the second-level subdomains are groups of first-level subdomains (the
    paper redistributes the coarse operator of 256 subdomains onto 4
    processes): the p_i coarse unknowns of subdomain i all belong to the
    second-level subdomain groups[i];
  * the graph of E used for the second-level overlap is the block pattern
    of E: a p_i x p_j block for every pair of subdomains whose non-overlapping
    sets are coupled in A (A(Omega_Ii, Omega_Ij) has a structural non-zero),
    plus the diagonal blocks, every entry of such a block kept (numerical
    zeros included);
  * the coarse unknowns of a first-level subdomain are ordered as its
    selected eigenvectors (A_II-orthonormal, Eq. (Zi)), subdomains in order;
  * the inner solve starts from e = 0 and stops at |g_{j+1}| <= 1e-4 ||c||_2
    or after its iteration limit, without error (an inexact coarse solve);
    the outer solver is flexible because the preconditioner then varies from
    one application to the next.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import amdd_oracle as O


def coupled_pairs(As: sp.csr_matrix, part: np.ndarray) -> set:
    """Pairs (i, j), i != j, of subdomains with A(Omega_Ii, Omega_Ij) != 0
    (structural non-zeros)."""
    C = As.tocoo()
    pi, pj = np.asarray(part)[C.row], np.asarray(part)[C.col]
    m = pi != pj
    return set(zip(pi[m].tolist(), pj[m].tolist()))


def coarse_matrix_blocks(S: O.Setup, part: np.ndarray) -> sp.csr_matrix:
    """E = R_0 A R_0^T as a sparse matrix with the block pattern: every entry
    of E_ij for i == j or (i, j) coupled in A, for subdomains with p > 0."""
    N = len(S.subs)
    off = np.concatenate([[0], np.cumsum([s.p for s in S.subs])])
    pairs = coupled_pairs(S.A, part)
    rows, cols, vals = [], [], []
    for i in range(N):
        for j in range(N):
            if S.subs[i].p == 0 or S.subs[j].p == 0:
                continue
            if i != j and (i, j) not in pairs:
                continue
            r = np.arange(off[i], off[i + 1])
            c = np.arange(off[j], off[j + 1])
            rr, cc = np.meshgrid(r, c, indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(S.E[off[i]:off[i + 1], off[j]:off[j + 1]].ravel())
    n = int(off[-1])
    if not rows:
        return sp.csr_matrix((n, n))
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return M.tocsr()


def coarse_partition(S: O.Setup, groups: np.ndarray) -> np.ndarray:
    """Second-level partition of the coarse unknowns: those of first-level
    subdomain i go to groups[i]."""
    return np.concatenate([np.full(s.p, groups[i], np.int32) for i, s in enumerate(S.subs)]) \
        if S.nC else np.zeros(0, np.int32)


@dataclass
class Multilevel:
    S1: O.Setup                 # first level (on A)
    S2: O.Setup                 # second level (on E)
    E: sp.csr_matrix            # E with the block pattern
    inner_rtol: float = 1e-4
    inner_restart: int = 30
    inner_maxit: int = 100
    inner_its: list = field(default_factory=list)


def setup(A, part, N: int, overlap: int, tau: float, groups, N2: int, overlap2: int, tau2: float,
          eps: float = O.EPS, inner_rtol: float = 1e-4, inner_restart: int = 30,
          inner_maxit: int = 100) -> Multilevel:
    """First level on A as in the two-level setup; then the same setup on the
    block-pattern E with the grouped partition of its unknowns."""
    S1 = O.setup(A, part, N, overlap, tau, eps)
    E = coarse_matrix_blocks(S1, np.asarray(part))
    part2 = coarse_partition(S1, np.asarray(groups))
    S2 = O.setup(E, part2, N2, overlap2, tau2, eps)
    return Multilevel(S1, S2, E, inner_rtol, inner_restart, inner_maxit)


def coarse_solve(ML: Multilevel, c: np.ndarray) -> np.ndarray:
    """Inexact C_00^{-1} c: right-preconditioned GMRES on E e = c with the
    deflated two-level method of the second level, e0 = 0."""
    e, its, _ = O.gmres(ML.E, c, lambda v: O.apply_deflated(ML.S2, v), restart=ML.inner_restart,
                        rtol=ML.inner_rtol, maxit=ML.inner_maxit)
    ML.inner_its.append(its)
    return e


def apply_deflated(ML: Multilevel, r: np.ndarray) -> np.ndarray:
    """Sec. 4.1 deflated form on the first level with the inexact coarse
    solve: zc = R_0^T C_00^{-1} R_0 r, z = zc + M_RAS (r - A zc)."""
    S = ML.S1
    if S.nC == 0:
        return O.apply_ras(S, r)
    zc = S.W @ coarse_solve(ML, S.W.T @ r)
    return zc + O.apply_ras(S, r - S.A @ zc)


def solve(ML: Multilevel, b: np.ndarray, restart: int = 30, rtol: float = 1e-8, maxit: int = 1000):
    """Outer flexible GMRES(restart) (the oracle's GMRES keeps the
    preconditioned vectors, so it is flexible) with the multilevel
    preconditioner; returns (x, iterations, history)."""
    return O.gmres(ML.S1.A, b, lambda v: apply_deflated(ML, v), restart=restart, rtol=rtol, maxit=maxit)
