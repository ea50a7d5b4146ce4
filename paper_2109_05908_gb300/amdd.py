"""Thin ctypes binding of libamdd (include/amdd.h): argument marshalling only.

Every numerical step runs inside the CUDA library.  Device buffers are passed
as raw pointers (for example `tensor.data_ptr()` of CUDA torch tensors, which
is how the tests and the benchmark provide device memory and streams).  The
library must be built (`build.build()`); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamdd.so")

AMDD_OK = 0
STATUS_NAMES = {0: "AMDD_OK", 1: "AMDD_ERR_INVALID", 2: "AMDD_ERR_NOT_SPD", 3: "AMDD_ERR_NOCONV",
                4: "AMDD_ERR_OOM", 5: "AMDD_ERR_TIMEOUT", 6: "AMDD_ERR_CUDA", 7: "AMDD_ERR_EIG_NOCONV"}


class amdd_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p)]


class amdd_proposal(C.Structure):
    _fields_ = [("weights", C.c_void_p), ("mean", C.c_void_p), ("sd", C.c_void_p)]


class amdd_opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_sweeps", C.c_int32), ("profile", C.c_int32),
                ("precision", C.c_int32), ("profile_classes", C.c_uint32), ("eig_solver", C.c_int32),
                ("keep_proposal_data", C.c_int32), ("proposal", C.POINTER(amdd_proposal)),
                ("keep_coarse_matrix", C.c_int32), ("reserved", C.c_int32), ("tie_band", C.c_double),
                ("use_graphs", C.c_int32), ("autotune", C.c_int32), ("mem_budget", C.c_size_t),
                ("tensor_cores", C.c_int32), ("local_solver", C.c_int32),
                ("jacobi_inner_sweeps", C.c_int32)]


MLP_NPARAM = 140032
PROP_NF = 32
PROP_NB = 16


class amdd_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("solve_ms", C.c_double), ("ritz_min", C.c_double),
                ("ritz_max", C.c_double), ("cond_est", C.c_double)]


class amdd_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("N", C.c_int32), ("overlap", C.c_int32), ("tau", C.c_double),
                ("n_C", C.c_int64), ("sum_ni", C.c_int64), ("sum_nti", C.c_int64), ("max_ni", C.c_int32),
                ("max_nti", C.c_int32), ("sweeps_svd", C.c_int32), ("sweeps_eig", C.c_int32),
                ("setup_ms", C.c_double), ("rotations_svd", C.c_int64), ("rotations_eig", C.c_int64),
                ("sweeps_svd32", C.c_int32), ("sweeps_eig32", C.c_int32), ("precision", C.c_int32),
                ("eps", C.c_double), ("n_partial", C.c_int32), ("lobpcg_subdomains", C.c_int32),
                ("lobpcg_fallbacks", C.c_int32), ("lobpcg_iters_max", C.c_int32),
                ("lobpcg_iters_total", C.c_int64), ("robust_schur", C.c_int32), ("levels", C.c_int32),
                ("inner_iterations_max", C.c_int32),
                ("inner_solves", C.c_int64), ("inner_iterations", C.c_int64), ("n_tied", C.c_int32),
                ("n_below_one", C.c_int32), ("device_bytes_peak", C.c_int64), ("graph_solves", C.c_int64),
                ("tuned_buckets", C.c_int64), ("sparse_local_nnz", C.c_int64),
                ("pair_stats", C.c_int64 * 10)]


class AmddError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({status_str(status)})")
        self.status = status


_lib = None

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "amdd_opts_default": (C.c_int, [C.POINTER(amdd_opts)]),
    "amdd_spmv": (C.c_int, [C.POINTER(amdd_csr), C.c_void_p, C.c_void_p, C.c_void_p]),
    "amdd_wait_selftest": (C.c_int, [C.c_int32, C.c_void_p]),
    "amdd_gemm_f32": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_void_p, C.c_int32, C.c_int32, C.c_float, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_void_p]),
    "amdd_setup": (C.c_int, [C.POINTER(amdd_csr), C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                             C.POINTER(amdd_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "amdd_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "amdd_pcg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                 C.POINTER(amdd_stats)]),
    "amdd_apply_form": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "amdd_gmres_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                   C.c_double, C.c_int32, C.POINTER(amdd_stats)]),
    "amdd_get_info": (C.c_int, [C.c_void_p, C.POINTER(amdd_info)]),
    "amdd_setup_next_level": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double,
                                        C.POINTER(amdd_opts), C.c_int32, C.c_double, C.c_int32]),
    "amdd_next_level": (C.c_void_p, [C.c_void_p]),
    "amdd_proposal_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.POINTER(C.c_int32)]),
    "amdd_get_eig_iterations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "amdd_mlp_sizes": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "amdd_mlp_feature_stats": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "amdd_mlp_normalize": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "amdd_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "amdd_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                      C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "amdd_mlp_round_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "amdd_lanczos_extremes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "amdd_get_subdomain": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "amdd_get_eigenvalues": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "amdd_get_singular_values": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                           C.POINTER(C.c_int32)]),
    "amdd_get_coarse_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32)]),
    "amdd_nd_order": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_int64)]),
    "amdd_overlap_sets": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "amdd_get_profile": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "amdd_reset_profile": (C.c_int, [C.c_void_p]),
    "amdd_true_residual_noalloc": (C.c_int, [C.POINTER(amdd_csr), C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "amdd_destroy": (None, [C.c_void_p]),
    "amdd_status_str": (C.c_char_p, [C.c_int]),
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libamdd.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(st: int) -> str:
    return lib().amdd_status_str(int(st)).decode()


def _check(st: int, where: str, allow=()):
    if st != AMDD_OK and st not in allow:
        raise AmddError(st, where)
    return st


def opts_default() -> amdd_opts:
    o = amdd_opts()
    _check(lib().amdd_opts_default(C.byref(o)), "amdd_opts_default")
    return o


def make_csr(n: int, nnz: int, rowptr_ptr: int, colind_ptr: int, val_ptr: int) -> amdd_csr:
    return amdd_csr(n, nnz, rowptr_ptr, colind_ptr, val_ptr)


def gemm_f32(m: int, n: int, k: int, alpha: float, a_ptr: int, lda: int, ta: int, b_ptr: int, ldb: int, tb: int,
             beta: float, c_ptr: int, ldc: int, tensor_cores: int = 1, stream: int = 0) -> None:
    """C = alpha op(A) op(B) + beta C in FP32 through amdd_gemm_f32."""
    _check(lib().amdd_gemm_f32(m, n, k, alpha, a_ptr, lda, ta, b_ptr, ldb, tb, beta, c_ptr, ldc, tensor_cores,
                               stream), "amdd_gemm_f32")


def wait_selftest(set_flag: bool, stream: int = 0) -> None:
    """Bounded device wait on a flag that is set (returns) or never set
    (raises AmddError with AMDD_ERR_TIMEOUT)."""
    _check(lib().amdd_wait_selftest(1 if set_flag else 0, stream), "amdd_wait_selftest")


def spmv(A: amdd_csr, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
    _check(lib().amdd_spmv(C.byref(A), x_ptr, y_ptr, stream), "amdd_spmv")


def setup(A: amdd_csr, part_ptr: int, N: int, overlap: int, tau: float, opts: amdd_opts | None = None,
          stream: int = 0) -> int:
    h = C.c_void_p()
    st = lib().amdd_setup(C.byref(A), part_ptr, N, overlap, float(tau), C.byref(opts) if opts else None,
                          stream, C.byref(h))
    _check(st, "amdd_setup")
    return h.value


def apply(h: int, r_ptr: int, z_ptr: int, nrhs: int = 1) -> None:
    _check(lib().amdd_apply(h, r_ptr, z_ptr, nrhs), "amdd_apply")


def pcg_solve(h: int, b_ptr: int, x_ptr: int, nrhs: int = 1, rtol: float = 1e-8, maxit: int = 1000,
              allow_noconv: bool = False) -> amdd_stats:
    s = amdd_stats()
    _check(lib().amdd_pcg_solve(h, b_ptr, x_ptr, nrhs, float(rtol), maxit, C.byref(s)), "amdd_pcg_solve",
           allow=(3,) if allow_noconv else ())
    return s


FORM_ADDITIVE, FORM_DEFLATED, FORM_RAS, FORM_ASM = 0, 1, 2, 3
# amdd_opts.eig_solver values
EIG_DENSE, EIG_LOBPCG, EIG_LEARNED, EIG_MATRIX_FREE = 0, 1, 2, 3
GMRES_MAX_RESTART = 64


def apply_form(h: int, form: int, r_ptr: int, z_ptr: int, nrhs: int = 1) -> None:
    _check(lib().amdd_apply_form(h, form, r_ptr, z_ptr, nrhs), "amdd_apply_form")


def gmres_solve(h: int, form: int, b_ptr: int, x_ptr: int, nrhs: int = 1, restart: int = 30, rtol: float = 1e-8,
                maxit: int = 1000, allow_noconv: bool = False) -> amdd_stats:
    s = amdd_stats()
    _check(lib().amdd_gmres_solve(h, form, b_ptr, x_ptr, nrhs, restart, float(rtol), maxit, C.byref(s)),
           "amdd_gmres_solve", allow=(3,) if allow_noconv else ())
    return s


def setup_next_level(h: int, groups, N2: int, overlap2: int, tau2: float, opts2: amdd_opts | None = None,
                     inner_restart: int = 30, inner_rtol: float = 1e-4, inner_maxit: int = 100) -> int:
    """Attach a second level built on the coarse matrix of h (host int32
    groups[N]); returns the second-level handle (owned by h)."""
    import numpy as np
    g = np.ascontiguousarray(groups, dtype=np.int32)
    _check(lib().amdd_setup_next_level(h, g.ctypes.data, N2, overlap2, float(tau2),
                                       C.byref(opts2) if opts2 else None, inner_restart, float(inner_rtol),
                                       inner_maxit), "amdd_setup_next_level")
    return lib().amdd_next_level(h)


def next_level(h: int):
    return lib().amdd_next_level(h)


def get_info(h: int) -> amdd_info:
    info = amdd_info()
    _check(lib().amdd_get_info(h, C.byref(info)), "amdd_get_info")
    return info


def get_subdomain(h: int, i: int):
    a, b, c, p = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().amdd_get_subdomain(h, i, C.byref(a), C.byref(b), C.byref(c), C.byref(p)), "amdd_get_subdomain")
    return a.value, b.value, c.value, p.value


def get_eigenvalues(h: int, i: int):
    import numpy as np
    cnt = C.c_int32()
    _check(lib().amdd_get_eigenvalues(h, i, None, 0, C.byref(cnt)), "amdd_get_eigenvalues")
    out = np.empty(cnt.value, dtype=np.float64)
    _check(lib().amdd_get_eigenvalues(h, i, out.ctypes.data, cnt.value, C.byref(cnt)), "amdd_get_eigenvalues")
    return out


def get_singular_values(h: int, i: int):
    import numpy as np
    cnt = C.c_int32()
    _check(lib().amdd_get_singular_values(h, i, None, 0, C.byref(cnt)), "amdd_get_singular_values")
    out = np.empty(cnt.value, dtype=np.float64)
    _check(lib().amdd_get_singular_values(h, i, out.ctypes.data, cnt.value, C.byref(cnt)),
           "amdd_get_singular_values")
    return out


def get_coarse_block(h: int, i: int):
    import numpy as np
    p, nI = C.c_int32(), C.c_int32()
    _check(lib().amdd_get_coarse_block(h, i, None, 0, C.byref(p), C.byref(nI)), "amdd_get_coarse_block")
    out = np.empty((p.value, nI.value), dtype=np.float64)
    if out.size:
        _check(lib().amdd_get_coarse_block(h, i, out.ctypes.data, out.size, C.byref(p), C.byref(nI)),
               "amdd_get_coarse_block")
    return out


def nd_order(n, rowptr, colind, leaf: int = 64):
    """Host-only nested-dissection order and symbolic Cholesky factor of a
    host CSR pattern; returns (perm, parent, colcount, nnzL)."""
    import numpy as np
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    perm = np.empty(n, np.int32)
    parent = np.empty(n, np.int32)
    cc = np.empty(n, np.int64)
    nnz = C.c_int64()
    _check(lib().amdd_nd_order(n, rowptr.ctypes.data, colind.ctypes.data, leaf, perm.ctypes.data, parent.ctypes.data,
                               cc.ctypes.data, C.byref(nnz)), "amdd_nd_order")
    return perm, parent, cc, nnz.value


def overlap_sets(n, rowptr, colind, part, i: int, overlap: int):
    """Host-only Sec. 2.1 sets of subdomain i from host numpy arrays
    (rowptr int64, colind int32, part int32); returns (I, G, D)."""
    import numpy as np
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    args = (n, rowptr.ctypes.data, colind.ctypes.data, part.ctypes.data, i, overlap)
    _check(lib().amdd_overlap_sets(*args, None, 0, None, 0, None, 0, C.byref(a), C.byref(b), C.byref(c)),
           "amdd_overlap_sets")
    I = np.empty(a.value, np.int32)
    G = np.empty(b.value, np.int32)
    D = np.empty(c.value, np.int32)
    _check(lib().amdd_overlap_sets(*args, I.ctypes.data, a.value, G.ctypes.data, b.value, D.ctypes.data, c.value,
                                   C.byref(a), C.byref(b), C.byref(c)), "amdd_overlap_sets")
    return I, G, D


def proposal_export(h: int):
    """(features (count x 32), target projectors (count x 16 x 16), subdomain
    indices) of a handle built with keep_proposal_data = 1 (host numpy)."""
    import numpy as np
    cnt = C.c_int32()
    _check(lib().amdd_proposal_export(h, None, None, None, 0, C.byref(cnt)), "amdd_proposal_export")
    n = cnt.value
    feat = np.empty((n, PROP_NF), np.float32)
    tgt = np.empty((n, PROP_NB, PROP_NB), np.float32)
    sub = np.empty(n, np.int32)
    if n:
        _check(lib().amdd_proposal_export(h, feat.ctypes.data, tgt.ctypes.data, sub.ctypes.data, n, C.byref(cnt)),
               "amdd_proposal_export")
    return feat, tgt, sub


def eig_iterations(h: int, N: int):
    import numpy as np
    out = np.empty(N, np.int32)
    _check(lib().amdd_get_eig_iterations(h, out.ctypes.data, N), "amdd_get_eig_iterations")
    return out


def mlp_sizes(n: int):
    a, b = C.c_int64(), C.c_int64()
    _check(lib().amdd_mlp_sizes(n, C.byref(a), C.byref(b)), "amdd_mlp_sizes")
    return a.value, b.value


def mlp_feature_stats(feat_ptr: int, n: int, mean_ptr: int, sd_ptr: int, stream: int = 0) -> None:
    _check(lib().amdd_mlp_feature_stats(feat_ptr, n, mean_ptr, sd_ptr, stream), "amdd_mlp_feature_stats")


def mlp_normalize(feat_ptr: int, mean_ptr: int, sd_ptr: int, n: int, x_ptr: int, stream: int = 0) -> None:
    _check(lib().amdd_mlp_normalize(feat_ptr, mean_ptr, sd_ptr, n, x_ptr, stream), "amdd_mlp_normalize")


def mlp_forward(wb_ptr: int, x_ptr: int, n: int, q_ptr: int, work_ptr: int, stream: int = 0) -> None:
    _check(lib().amdd_mlp_forward(wb_ptr, x_ptr, n, q_ptr, work_ptr, stream), "amdd_mlp_forward")


def mlp_train_step(w_ptr, wb_ptr, m_ptr, v_ptr, t: int, lr: float, x_ptr, qt_ptr, n: int, grad_ptr, work_ptr,
                   loss_ptr, stream: int = 0) -> None:
    _check(lib().amdd_mlp_train_step(w_ptr, wb_ptr, m_ptr, v_ptr, t, float(lr), x_ptr, qt_ptr, n, grad_ptr,
                                     work_ptr, loss_ptr, stream), "amdd_mlp_train_step")


def mlp_round_bf16(w_ptr: int, wb_ptr: int, n: int, stream: int = 0) -> None:
    _check(lib().amdd_mlp_round_bf16(w_ptr, wb_ptr, n, stream), "amdd_mlp_round_bf16")


def lanczos_extremes(alpha, beta):
    """Host-only extreme eigenvalues of the PCG Lanczos tridiagonal from the
    step lengths alpha[k] and ratios beta[k-1]; returns (lo, hi)."""
    import numpy as np
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    _check(lib().amdd_lanczos_extremes(a.ctypes.data if a.size else None, b.ctypes.data if b.size else None,
                                       int(a.size), C.byref(lo), C.byref(hi)), "amdd_lanczos_extremes")
    return lo.value, hi.value


PROF_CLASSES = 27


def get_profile(h: int):
    """List of dicts (name, launches, ms, flops, bytes), one per kernel class."""
    out = []
    for k in range(PROF_CLASSES):
        name, n, ms, fl, by = C.c_char_p(), C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        _check(lib().amdd_get_profile(h, k, C.byref(name), C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)),
               "amdd_get_profile")
        out.append(dict(name=name.value.decode(), launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value))
    return out


def reset_profile(h: int) -> None:
    _check(lib().amdd_reset_profile(h), "amdd_reset_profile")


NOALLOC_MAX_N = 524288


def true_residual_noalloc(A: amdd_csr, b_ptr: int, x_ptr: int, stream: int = 0):
    """(||b - A x||_2, ||b||_2) through the allocation-free entry point."""
    out = (C.c_double * 2)()
    _check(lib().amdd_true_residual_noalloc(C.byref(A), b_ptr, x_ptr, C.cast(out, C.c_void_p), stream),
           "amdd_true_residual_noalloc")
    return out[0], out[1]


def destroy(h: int) -> None:
    if h:
        lib().amdd_destroy(h)
