/*
 * amdd.h -- C ABI of a GB300 (sm_103a) implementation of the fully algebraic
 * two-level overlapping Schwarz preconditioner for sparse SPD systems of
 * Al Daas & Jolivet, "A robust algebraic multilevel domain decomposition
 * preconditioner for sparse symmetric positive definite matrices"
 * (arXiv 2109.05908).
 *
 * Problem (Sec. 1): solve A x = b, A n x n sparse SPD.
 * Setup (Sec. 2.1, Eq. (Xi), Sec. 3.2, Eq. (tildeA), Eq. (Zi)): for each of
 * the N non-overlapping subdomains Omega_Ii given by `part`, build the
 * overlap Omega_Gi (graph distance 1..overlap), the extension Omega_Di
 * (distance overlap+1), the local block row X_i = R_i A tilde R_i^T, its
 * regularised square root Abar_ii, the local eigenproblem
 * D_i A_ii D_i u = lambda tilde A_ii u with Boolean D_i, and keep the
 * eigenvectors with lambda > 1/tau as the coarse block Z_i.  Then assemble
 * and factor the coarse matrix E = R_0 A R_0^T, R_0^T = [R_i^T D_i Z_i].
 * Apply (Eq. (two_level_schwarz)):
 *     z = R_0^T E^{-1} R_0 r + sum_i R_i^T A_ii^{-1} R_i r.
 * Solve: preconditioned conjugate gradient with that z.
 *
 * Conventions for every entry point:
 *   - Pointers documented as "device" must be CUDA device pointers valid on
 *     the current device; "host" pointers are ordinary host memory.
 *   - The caller owns every buffer it passes; the library never frees or
 *     retains caller memory past the call.  A handle owns every device and
 *     host buffer it allocates, released by amdd_destroy.
 *   - All GPU work of a handle is issued on the CUDA stream given to
 *     amdd_setup (NULL = legacy default stream).  Calls return after the work
 *     they issued has completed (they synchronise that stream), so results in
 *     caller buffers are ready on return.
 *   - Every call returns a status and never aborts the process.  Device-side
 *     errors (a non-positive Cholesky pivot, an eigensolver that did not
 *     converge) are latched and returned by the call that detects them.
 *   - Not thread-safe per handle: one host thread at a time per handle.
 */
#ifndef AMDD_H
#define AMDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMDD_OK = 0,
    AMDD_ERR_INVALID = 1,     /* bad argument, size or partition                  */
    AMDD_ERR_NOT_SPD = 2,     /* a Cholesky pivot <= 0 (A_ii or E not SPD)         */
    AMDD_ERR_NOCONV = 3,      /* PCG reached maxit before the tolerance            */
    AMDD_ERR_OOM = 4,         /* a device or host allocation failed                */
    AMDD_ERR_TIMEOUT = 5,     /* a bounded device wait (tensor cores, Jacobi sweep) gave up */
    AMDD_ERR_CUDA = 6,        /* any other CUDA runtime error                      */
    AMDD_ERR_EIG_NOCONV = 7   /* a Jacobi eigensolver hit its sweep limit          */
} amdd_status;

typedef struct amdd_handle amdd_handle;

/* Square sparse matrix in CSR form, full symmetric pattern, DEVICE pointers.
 * rowptr[n+1] (int64), colind[nnz] (int32, ascending in each row), val[nnz]. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* rowptr;
    const int32_t* colind;
    const double* val;
} amdd_csr;

/* A trained proposal network for the learned warm start of the local
 * eigensolve (no counterpart in the paper: an accelerator of the eigensolve
 * of eq. (Zi) whose results are accepted only if they pass the same checks
 * as those of the plain eigensolver).  Device pointers, FP32, owned by the
 * caller and read during amdd_setup only:
 *   weights  AMDD_MLP_NPARAM values rounded to bfloat16 (amdd_mlp_train_step
 *            keeps such a copy), layout W1 (32 x 256), b1 (256), W2
 *            (256 x 256), b2, W3 (256 x 256), b3, matrices row-major;
 *   mean, sd the 32 feature means and standard deviations (sd > 0) the
 *            network was trained with. */
typedef struct {
    const float* weights;
    const float* mean;
    const float* sd;
} amdd_proposal;

#define AMDD_MLP_NPARAM 140032
#define AMDD_PROP_NF 32
#define AMDD_PROP_NB 16

typedef struct {
    double eps;           /* shift of Remark 3.2 / Sec. 3.2: Abar += sigma_1*eps*I; default 2^-52 */
    int32_t max_sweeps;   /* sweep limit of the one-sided Jacobi solvers; default 60               */
    int32_t profile;      /* 1: time every kernel launch of the handle with CUDA events (see
                             amdd_get_profile); default 0                                           */
    int32_t precision;    /* 0: plain FP64 (default).
                             1: mixed form: the local work (local Cholesky factors and solves, SVD
                             of X_i, splitting, eq. (Zi)) in FP32 with FP32 accumulation; E, its
                             factor, the coarse solve and PCG in FP64.  Sec. 3.2 takes eps as the
                             machine precision of the arithmetic, so the FP32 stage uses
                             max(eps, 2^-23) (amdd_info.eps reports it).
                             2: mixed form with an FP64 splitting: the SVD of X_i, Abar_ii and its
                             Schur complement in FP64 with eps as given; the local factors and
                             solves, T and the eigensolve of eq. (Zi) in FP32; E and PCG in FP64 */
    uint32_t profile_classes; /* with profile = 1: bit k set times kernel class k only (classes as
                             numbered by amdd_get_profile); 0 times every class; default 0         */
    int32_t eig_solver;   /* eigenvectors of eq. (Zi) when the selection is partial: 0 dense one-sided
                             Jacobi on [T | I] (default); 1 block LOBPCG from counter-based random
                             rows; 2 block LOBPCG from the learned proposal (needs `proposal`).
                             A LOBPCG result is accepted only if every wanted residual is within
                             the tolerance and its Ritz values match the bisection eigenvalues;
                             otherwise that subdomain takes the dense path.
                             3: matrix-free eigensolve (Sec. 3.2, eq. (invAii)): neither Abar_ii,
                             its Schur complement nor T_i is formed; block LOBPCG finds the largest
                             eigenpairs of K_i = L_A^T (Abar_ii^{-1})_II L_A with (Abar_ii^{-1})_II
                             applied from the SVD of X_i, the block doubling until its last
                             converged eigenvalue is at most 1/tau.  Needs precision = 0,
                             eps >= 2^-30 (below that the two terms of eq. (invAii) cancel in FP64
                             and the eigenvalues near 1/tau lose all accuracy) and
                             keep_proposal_data = 0; otherwise AMDD_ERR_INVALID                   */
    int32_t keep_proposal_data; /* 1: keep the features and Krylov bases of the partially selected
                             subdomains for amdd_proposal_export                                     */
    const amdd_proposal* proposal; /* the network of eig_solver = 2 (NULL otherwise)                */
    int32_t keep_coarse_matrix; /* 1: keep a copy of the coarse matrix E (block pattern, see
                             amdd_setup_next_level) for a next level; default 0                     */
    int32_t reserved;     /* must be zero                                                          */
    double tie_band;      /* eigenvalues of eq. (Zi) within a relative band of the threshold,
                             |lambda tau - 1| <= tie_band, are counted in amdd_info.n_tied: the
                             selection lambda > 1/tau of eq. (Zi) is unchanged, but two correct
                             eigensolvers may disagree on such an eigenvalue; default 1e-10, >= 0 */
    int32_t use_graphs;   /* 1: amdd_pcg_solve replays its iterations as CUDA graphs, several per
                             host synchronisation, and stops them on the device once converged
                             (same arithmetic and results as 0); 0: one launch sequence and one
                             host synchronisation per iteration; default 1                        */
    int32_t autotune;     /* 1: the batched GEMM tile (16, 32 or 64) is measured once per size
                             bucket and process on the first batch that can be rerun, and the
                             fastest kept (the tile size never changes a result, only its time);
                             0: a fixed rule on the launch size; default 1                          */
    size_t mem_budget;    /* largest number of device bytes the handle may hold at once, setup
                             temporaries included; an allocation beyond it fails with
                             AMDD_ERR_OOM before it is made (amdd_info.device_bytes_peak reports
                             what a setup used); 0 (default): no limit                             */
    int32_t tensor_cores; /* 1: FP32 batched GEMMs of at least 16 output tiles of 128 x 128 (the
                             mixed form's local products), and the Gram matrices and rotations of
                             the FP32 block-pair Jacobi, run on the tcgen05 tensor cores in TF32
                             with the 3xTF32 split (hi*hi + hi*lo + lo*hi, FP32 accumulation), whose
                             error is of the order of an FP32 multiply-add loop's; 0: CUDA-core FMA;
                             default 1                                                              */
    int32_t local_solver; /* local solves of the Schwarz methods (Sec. 4.1: exact local Cholesky):
                             0: the explicit inverse factors L_i^{-1}, L_i^{-T} (dense triangles);
                             1: sparse Cholesky factors in a nested-dissection order (the same exact
                             factor of the permuted A_ii, with the symbolic fill only), solved by
                             forward and backward substitution with each factor staged in shared
                             memory; AMDD_ERR_INVALID if a factor does not fit (about 200 KB);
                             2: 1 where every factor fits and holds at most a quarter of its dense
                             triangle, else 0; default 0                                           */
    int32_t jacobi_inner_sweeps; /* block-pair Jacobi (matrices whose rows exceed shared memory):
                             at most this many sweeps of the 64 x 64 eigensolve per visit of a
                             block pair (the outer sweeps repeat until every pair passes the
                             stopping test, so the result meets the same test); 0 (default): 1
                             (one inner sweep, measured fastest: the outer sweep count did not
                             grow); AMDD_ERR_INVALID above 64                                      */
} amdd_opts;

typedef struct {
    int32_t iterations;         /* PCG iterations performed (first right-hand side)          */
    int32_t converged;          /* 1 if ||r_k|| <= rtol ||b|| was reached                    */
    double rel_residual;        /* recursive residual ||r_k|| / ||b|| at exit                */
    double true_rel_residual;   /* ||b - A x|| / ||b|| recomputed at exit                    */
    double solve_ms;            /* wall time of the call                                     */
    double ritz_min;            /* extreme eigenvalues of the Lanczos tridiagonal built from  */
    double ritz_max;            /* the PCG step lengths alpha_k and ratios beta_k (first     */
    double cond_est;            /* right-hand side): Ritz values of M^{-1} A, inside its     */
                                /* spectrum; cond_est = ritz_max / ritz_min, the estimate    */
                                /* checked against the bound of Sec. 3.2 (NaN: no step)      */
} amdd_stats;

typedef struct {
    int64_t n;             /* order of A                                   */
    int32_t N;             /* number of subdomains                         */
    int32_t overlap;       /* overlap layers                               */
    double tau;            /* prescribed bound parameter of eq. (Zi)       */
    int64_t n_C;           /* coarse dimension sum_i p_i                   */
    int64_t sum_ni;        /* sum of |Omega_i|                             */
    int64_t sum_nti;       /* sum of |tilde Omega_i|                       */
    int32_t max_ni;        /* largest |Omega_i|                            */
    int32_t max_nti;       /* largest |tilde Omega_i|                      */
    int32_t sweeps_svd;    /* largest Jacobi sweep count for the SVD of X_i */
    int32_t sweeps_eig;    /* largest Jacobi sweep count for eq. (Zi)      */
    double setup_ms;       /* wall time of amdd_setup                      */
    int64_t rotations_svd; /* plane rotations applied by the SVD solver    */
    int64_t rotations_eig; /* plane rotations applied by the eq. (Zi) solver */
    int32_t sweeps_svd32;  /* sweeps of the FP32 preconditioning stage (SVD) */
    int32_t sweeps_eig32;  /* sweeps of the FP32 preconditioning stage (eq. (Zi)) */
    int32_t precision;     /* 0 plain FP64, 1 or 2 mixed (see amdd_opts)     */
    double eps;            /* the eps of the splitting actually used       */
    int32_t n_partial;     /* subdomains whose selection is partial (0 < p_i < |Omega_Ii|) */
    int32_t lobpcg_subdomains; /* of those, eigenvectors accepted from LOBPCG (eig_solver 3:
                                  every subdomain, all solved by the matrix-free LOBPCG) */
    int32_t lobpcg_fallbacks;  /* LOBPCG results rejected (dense path taken)  */
    int32_t lobpcg_iters_max;  /* largest LOBPCG iteration count (eig_solver 3: of one block) */
    int64_t lobpcg_iters_total;/* sum of the LOBPCG iteration counts         */
    int32_t robust_schur;      /* subdomains whose Schur complement of the splitting was
                                  recomputed in the rounding-robust form (the Cholesky of
                                  its [Omega_Gi, Omega_Di] block lost definiteness)   */
    int32_t levels;            /* 1 + the levels attached by amdd_setup_next_level */
    int32_t inner_iterations_max; /* largest inner GMRES iteration count of a coarse solve */
    int64_t inner_solves;      /* coarse solves done by inner GMRES (since setup) */
    int64_t inner_iterations;  /* their total iteration count                  */
    int32_t n_tied;            /* eigenvalues of eq. (Zi) with |lambda tau - 1| <= tie_band */
    int32_t n_below_one;       /* eigenvalues of eq. (Zi) below 1 - 1e-6: without the shift
                                  sigma_1 eps every non-zero one is >= 1 with Boolean D_i; the
                                  shift lowers the bound to 1 / (1 + sigma_1 eps / lambda_min(A_II)),
                                  far below 1 for the FP32 splitting on high-contrast matrices */
    int64_t device_bytes_peak; /* largest device memory the handle has held (bytes) */
    int64_t graph_solves;      /* PCG solves whose iterations ran as one CUDA graph   */
    int64_t tuned_buckets;     /* GEMM size buckets measured by the autotuner in this process */
    int64_t sparse_local_nnz;  /* entries of the sparse local factors in use (0: dense inverse
                                  factors, see amdd_opts.local_solver)                      */
    int64_t pair_stats[10];     /* block-pair one-sided Jacobi (matrices whose rows exceed shared
                                  memory): pair tasks run, pairs rotated, SM clock cycles
                                  summed over CTAs of its three phases (Gram matrices, small
                                  eigensolves, rotation of the rows), inner sweeps; with the
                                  tensor-core sweep kernel also the cycles spent waiting for
                                  the previous round of a pair's row blocks, the summed
                                  lifetimes of its CTAs (cycles), the CTAs that ran at least one
                                  pair, and the CTAs launched                                  */
} amdd_info;

/* Symbolic phase of a sparse local Cholesky factorisation, on the host (no
 * GPU involved): a nested-dissection fill-reducing order of the symmetric
 * pattern of a HOST CSR graph (n, rowptr[n+1], colind[rowptr[n]]; the
 * pattern is symmetrised, the diagonal ignored) and the structure of the
 * Cholesky factor of P A P^T in that order.  Sec. 4.1 uses exact Cholesky
 * factorisations of the local matrices; a sparse factor in this order is
 * the same factor of the permuted matrix with far fewer entries than the
 * dense one.  Sets of at most `leaf` (>= 1) unknowns are not cut further.
 * Outputs (host arrays of n entries, the last three may be NULL):
 *   perm[k]      the unknown eliminated k-th (row k of P A P^T is row perm[k]);
 *   parent[k]    the elimination tree in the new numbering (-1 for a root);
 *   colcount[k]  entries of column k of the factor, the diagonal included;
 *   *nnzL        their sum.
 * AMDD_ERR_INVALID for a malformed graph or leaf < 1; AMDD_ERR_OOM if the
 * host allocation fails. */
amdd_status amdd_nd_order(int64_t n, const int64_t* rowptr, const int32_t* colind, int32_t leaf, int32_t* perm,
                          int32_t* parent, int64_t* colcount, int64_t* nnzL);

/* Fill `o` with the defaults (eps = 2^-52, max_sweeps = 60, tie_band = 1e-10,
 * use_graphs = 1, autotune = 1, tensor_cores = 1, everything else 0). */
amdd_status amdd_opts_default(amdd_opts* o);

/* C = alpha op(A) op(B) + beta C in FP32 (row-major; op(A) = A if ta = 0,
 * A^T if ta = 1; op(A) is m x k, op(B) is k x n), the dense block product the
 * setup's FP32 stage uses (Sec. 3.2: the splitting, the local Cholesky
 * factors and eq. (Zi)).  tensor_cores = 1: the tcgen05 kernel with the
 * 3xTF32 split (TF32 units, FP32 accumulation, error of the order of an FP32
 * multiply-add loop's); 0: CUDA-core FMA.  A, B, C are device pointers with
 * leading dimensions lda, ldb, ldc (>= the stored row length); work runs on
 * `stream` and is complete on return.  The call makes one small stream-ordered
 * allocation for its descriptors.  AMDD_ERR_INVALID on bad sizes or flags;
 * AMDD_ERR_TIMEOUT if a bounded wait of the tensor-core kernel gave up. */
amdd_status amdd_gemm_f32(int32_t m, int32_t n, int32_t k, float alpha, const float* A, int32_t lda, int32_t ta,
                          const float* B, int32_t ldb, int32_t tb, float beta, float* C, int32_t ldc,
                          int32_t tensor_cores, void* stream);

/* Check of the failure status of the library's bounded device waits (no
 * counterpart in the paper): the wait of the persistent block-pair Jacobi
 * sweep, run on its own for about 2 ms of SM clock on a device flag that is
 * 1 when `set_flag` is non-zero and stays 0 otherwise.  AMDD_OK when the flag
 * was set; AMDD_ERR_TIMEOUT when the wait gave up (the kernel returns normally
 * and the context stays usable); AMDD_ERR_OOM / AMDD_ERR_CUDA on allocation or
 * launch failure.  Allocates 8 bytes stream-ordered and synchronises `stream`. */
amdd_status amdd_wait_selftest(int32_t set_flag, void* stream);

/* y = A x (Sec. 1: the operator of A x = b).  A, x (length n) and y
 * (length n) are device pointers; y must not alias x.  Work is issued on
 * `stream` (cudaStream_t, may be NULL) and completed before return. */
amdd_status amdd_spmv(const amdd_csr* A, const double* x, double* y, void* stream);

/* Sec. 2.1 on the host, no GPU involved: the sets of subdomain i from a HOST
 * CSR graph (n, rowptr[n+1], colind[rowptr[n]]) and a HOST partition
 * part[n].  Omega_Ii = {j : part[j] == i}; Omega_Gi = unknowns at graph
 * distance 1..overlap from Omega_Ii; Omega_Di = unknowns at distance
 * overlap+1.  Each set is written ascending into the caller's host arrays
 * I[capI], G[capG], D[capD] (any may be NULL to query sizes only); the sizes
 * always go to *nI, *nG, *nD.  AMDD_ERR_INVALID if an array is too small or
 * the graph is malformed.  amdd_setup builds its sets with the same code. */
amdd_status amdd_overlap_sets(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* part,
                              int32_t i, int32_t overlap, int32_t* I, int32_t capI, int32_t* G, int32_t capG,
                              int32_t* D, int32_t capD, int32_t* nI, int32_t* nG, int32_t* nD);

/* Build the two-level preconditioner (Sec. 2.1, Eq. (Xi), Sec. 3.2,
 * Eq. (tildeA), Eq. (Zi), Eq. (two_level_schwarz)).
 *   A        device CSR of the SPD matrix (copied; the caller may free it after).
 *   part     device int32[n], part[j] in [0, N): the non-overlapping subdomain
 *            Omega_Ij of unknown j.  Every subdomain must be non-empty.
 *   N        number of subdomains (>= 1).
 *   overlap  number of overlap layers (>= 1).
 *   tau      > 0; the eigenvectors of eq. (Zi) with lambda > 1/tau are kept.
 *   opts     NULL for defaults.
 *   stream   cudaStream_t on which all work of the handle runs (NULL allowed).
 *   out      receives the handle (NULL on failure).
 * Errors: AMDD_ERR_INVALID (sizes, empty subdomain, part out of range, a NaN
 * or an infinity among the values of A),
 * AMDD_ERR_NOT_SPD (non-positive pivot in a local or the coarse Cholesky),
 * AMDD_ERR_EIG_NOCONV, AMDD_ERR_OOM, AMDD_ERR_CUDA. */
amdd_status amdd_setup(const amdd_csr* A, const int32_t* part, int32_t N, int32_t overlap,
                       double tau, const amdd_opts* opts, void* stream, amdd_handle** out);

/* z = M^{-1} r, Eq. (two_level_schwarz), for `nrhs` vectors.  r and z are
 * device pointers to nrhs contiguous vectors of length n (vector k at
 * offset k*n); z must not alias r. */
amdd_status amdd_apply(amdd_handle* h, const double* r, double* z, int32_t nrhs);

/* Preconditioned conjugate gradient on A x = b with M^{-1} of
 * Eq. (two_level_schwarz), for `nrhs` right-hand sides.  With nrhs > 1 the
 * right-hand sides are independent PCG iterations advanced together in
 * batches of up to 8: each batch shares one pass over A per SpMV and one pass
 * over the local and coarse factors per apply; a right-hand side that has
 * converged stops updating while the others go on.  b and x are device
 * pointers (nrhs contiguous vectors of length n); x holds the initial guess
 * on entry and the solution on return.  Stops when ||r_k||_2 <= rtol ||b||_2
 * (recursive residual) or after maxit iterations (AMDD_ERR_NOCONV).  A NaN or
 * an infinity in b or in the initial guess is AMDD_ERR_INVALID.  `stats`
 * (host, may be NULL) describes the first right-hand side. */
amdd_status amdd_pcg_solve(amdd_handle* h, const double* b, double* x, int32_t nrhs,
                           double rtol, int32_t maxit, amdd_stats* stats);

/* Preconditioner forms of amdd_apply_form and amdd_gmres_solve.
 *   AMDD_FORM_ADDITIVE  the additive two-level method, Eq. (two_level_schwarz):
 *                       z = R_0^T E^{-1} R_0 r + sum_i R_i^T A_ii^{-1} R_i r.
 *   AMDD_FORM_DEFLATED  the deflated two-level method of Sec. 4.1 with the
 *                       restricted one-level method and C = A:
 *                       zc = R_0^T E^{-1} R_0 r,  z = zc + M_RAS (r - A zc).
 *   AMDD_FORM_RAS       the one-level restricted additive Schwarz method of
 *                       Sec. 4.1: z = sum_i R_i^T D_i A_ii^{-1} R_i r (Boolean
 *                       D_i: every unknown takes the local solution of the
 *                       subdomain whose Omega_Ii holds it).
 *   AMDD_FORM_ASM       the one-level additive method of Sec. 2.1:
 *                       z = sum_i R_i^T A_ii^{-1} R_i r.
 * DEFLATED and RAS are not symmetric: use them with GMRES. */
typedef enum {
    AMDD_FORM_ADDITIVE = 0,
    AMDD_FORM_DEFLATED = 1,
    AMDD_FORM_RAS = 2,
    AMDD_FORM_ASM = 3
} amdd_form;

/* z = M^{-1} r for the preconditioner form `form` (amdd_form) of the
 * handle's setup, for `nrhs` vectors.  r and z are device pointers to nrhs
 * contiguous vectors of length n (vector k at offset k*n); z must not alias
 * r.  The local and coarse solves are those of amdd_apply (same precision).
 * AMDD_ERR_INVALID on a bad form or argument. */
amdd_status amdd_apply_form(amdd_handle* h, int32_t form, const double* r, double* z, int32_t nrhs);

/* Largest restart length of amdd_gmres_solve. */
#define AMDD_GMRES_MAX_RESTART 64

/* Right-preconditioned restarted GMRES(restart) (Saad and Schultz; the
 * Krylov method of the experiments of Sec. 4.1, there with restart 30) on
 * A x = b with the preconditioner form `form` (amdd_form), for `nrhs`
 * right-hand sides solved one after the other.  b and x are device pointers
 * (nrhs contiguous vectors of length n); x holds the initial guess on entry
 * and the solution on return.  Each cycle starts from r = b - A x; the
 * Arnoldi basis is orthogonalised by classical Gram-Schmidt applied twice.
 * Stops when the least-squares residual estimate |g_{j+1}| <= rtol ||b||_2
 * or after maxit Arnoldi steps in total (AMDD_ERR_NOCONV).  `stats` (host,
 * may be NULL) describes the first right-hand side: iterations = Arnoldi
 * steps, rel_residual = the estimate at exit, true_rel_residual recomputed;
 * ritz_min, ritz_max and cond_est are NaN.  The handle allocates
 * (restart + 1 + restart) n doubles of Krylov vectors on the first call (and
 * again when a later call asks for a longer restart).  AMDD_ERR_INVALID for
 * restart outside [1, AMDD_GMRES_MAX_RESTART], a bad form or argument. */
amdd_status amdd_gmres_solve(amdd_handle* h, int32_t form, const double* b, double* x, int32_t nrhs,
                             int32_t restart, double rtol, int32_t maxit, amdd_stats* stats);

/* Multilevel form (Sec. 3.2, last paragraph; Sec. 4.2): the same fully
 * algebraic construction applied to the coarse matrix E of handle h, whose
 * exact coarse solve is then replaced by an inexact one.  h must have been
 * set up with opts.keep_coarse_matrix = 1 and n_C > 0.
 *   groups   HOST int32[N] (N = subdomains of h): the coarse unknowns of
 *            subdomain i (its p_i selected eigenvectors) form part of
 *            second-level subdomain groups[i], in [0, N2); every group must
 *            hold at least one coarse unknown.
 *   N2, overlap2, tau2, opts2   as in amdd_setup, for the second level.
 *            The second level sees E as a sparse matrix with its block
 *            pattern: every entry of the p_i x p_j block E_ij for i == j or
 *            for subdomains whose non-overlapping sets are coupled in A
 *            (A(Omega_Ii, Omega_Ij) has a structural non-zero).
 *   inner_restart, inner_rtol, inner_maxit
 *            every later coarse solve of h (in amdd_apply, amdd_apply_form,
 *            amdd_pcg_solve, amdd_gmres_solve) is right-preconditioned
 *            GMRES(inner_restart) on E e = c from e = 0 with the deflated
 *            form of the second level, stopped at |g_{j+1}| <= inner_rtol
 *            ||c||_2 or after inner_maxit steps (no error: an inexact solve;
 *            the paper uses 30 and 1e-4).  The preconditioner of h then
 *            changes from one application to the next: solve with
 *            amdd_gmres_solve, which keeps the preconditioned vectors and so
 *            is the flexible GMRES of Sec. 4.2.
 * The second-level handle is owned by h (released by amdd_destroy(h)) and
 * can be inspected through amdd_next_level; calling this function again
 * replaces it.  h frees its copy of E afterwards.  Errors: AMDD_ERR_INVALID
 * (no kept E, bad groups or parameters), and those of amdd_setup. */
amdd_status amdd_setup_next_level(amdd_handle* h, const int32_t* groups, int32_t N2, int32_t overlap2,
                                  double tau2, const amdd_opts* opts2, int32_t inner_restart, double inner_rtol,
                                  int32_t inner_maxit);

/* The second-level handle attached by amdd_setup_next_level (borrowed,
 * owned by h), or NULL. */
amdd_handle* amdd_next_level(const amdd_handle* h);

/* Training data of the learned warm start (no counterpart in the paper)
 * from a handle built with opts.keep_proposal_data = 1: for each partially
 * selected subdomain, in subdomain order, its 32 features (feat, row-major
 * count x 32), the target 16 x 16 projector B^T Q Q^T B (target, count x 256;
 * B the orthonormal Krylov basis K_16(A_II, 1), Q an orthonormal basis of
 * the selected eigenvectors on Omega_Ii) and its subdomain index (sub).  Host
 * arrays of capacity cap (any may be NULL to query *count only).  Features
 * (definitions in the library's source): sizes and their ratios, statistics
 * of log diag(A_II), of log|off-diagonal entries|, of row degrees, of the
 * coupling to Omega_Gi and of diagonal dominance, ||A_II||_F, trace, sign
 * structure, p_i, tau.  AMDD_ERR_INVALID without the kept data. */
amdd_status amdd_proposal_export(const amdd_handle* h, float* feat, float* target, int32_t* sub, int32_t cap,
                                 int32_t* count);

/* Per-subdomain LOBPCG iteration counts into the host array iters[cap]
 * (cap >= N): >= 0 accepted from LOBPCG, -1 dense path, -2 selection not
 * partial.  With eig_solver 3 every subdomain with |Omega_Ii| > 0 has the
 * iteration count of its last (accepted) block; -2 for an empty one. */
amdd_status amdd_get_eig_iterations(const amdd_handle* h, int32_t* iters, int32_t cap);

/* The proposal network (no counterpart in the paper), trained on the GPU by
 * these kernels; all pointers are device pointers, work runs on `stream`
 * and is complete on return.  n = number of samples (rows).
 *   amdd_mlp_sizes: *nparam = AMDD_MLP_NPARAM, *nwork = floats of the `work`
 *     buffer amdd_mlp_forward / amdd_mlp_train_step need for n samples.
 *   amdd_mlp_feature_stats: mean[32] and sd[32] (population standard
 *     deviation, 1 where below 1e-6) of the columns of feat (n x 32), the
 *     standardisation the network is trained with.
 *   amdd_mlp_normalize: x = (feat - mean) / sd (n x 32).
 *   amdd_mlp_forward: q (n x 256) = the symmetrised outputs, as 16 x 16
 *     matrices, of the MLP 32 -> 256 -> 256 -> 256 (ReLU) with weights wb.
 *   amdd_mlp_train_step: forward with wb, loss = mean over samples of
 *     ||q - qt||_F^2 (written to *loss, a device float), its gradient in
 *     grad (AMDD_MLP_NPARAM), then, when lr > 0, one Adam step (beta1 0.9,
 *     beta2 0.999, eps 1e-8, step number t >= 1) on the FP32 master weights w
 *     with moments m, v, and wb = w rounded to bfloat16 (nearest, ties to
 *     even).  lr = 0 computes the gradient only.
 *   amdd_mlp_round_bf16: wb = w rounded to bfloat16 (n values). */
amdd_status amdd_mlp_sizes(int32_t n, int64_t* nparam, int64_t* nwork);
amdd_status amdd_mlp_feature_stats(const float* feat, int32_t n, float* mean, float* sd, void* stream);
amdd_status amdd_mlp_normalize(const float* feat, const float* mean, const float* sd, int32_t n, float* x,
                               void* stream);
amdd_status amdd_mlp_forward(const float* wb, const float* x, int32_t n, float* q, float* work, void* stream);
amdd_status amdd_mlp_train_step(float* w, float* wb, float* m, float* v, int32_t t, float lr, const float* x,
                                const float* qt, int32_t n, float* grad, float* work, float* loss, void* stream);
amdd_status amdd_mlp_round_bf16(const float* w, float* wb, int64_t n, void* stream);

/* Host-only, no GPU involved: the extreme eigenvalues of the Lanczos
 * tridiagonal of k PCG steps (the CG-Lanczos relation; Sec. 1 gives the CG
 * bound these Ritz values feed): T_11 = 1/alpha_1, T_jj = 1/alpha_j +
 * beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j, from the HOST
 * arrays alpha[k] (> 0) and beta[k-1] (>= 0; may be NULL for k <= 1).  Writes
 * *lo, *hi (NaN for k = 0).  AMDD_ERR_INVALID on a negative k or a
 * non-positive alpha / negative beta.  amdd_pcg_solve reports the same
 * values in amdd_stats. */
amdd_status amdd_lanczos_extremes(const double* alpha, const double* beta, int32_t k, double* lo, double* hi);

/* Sizes and counters of a handle (host struct). */
amdd_status amdd_get_info(const amdd_handle* h, amdd_info* info);

/* Sizes of subdomain i: |Omega_Ii|, |Omega_Gi|, |Omega_Di| and p_i (host out). */
amdd_status amdd_get_subdomain(const amdd_handle* h, int32_t i, int32_t* nI, int32_t* nG,
                               int32_t* nD, int32_t* p);

/* The |Omega_Ii| non-zero eigenvalues of eq. (Zi) of subdomain i, descending,
 * into the host array lam[cap]; +inf marks an eps-cluster eigenvalue whose
 * computed reciprocal was not positive.  With the matrix-free eigensolve
 * (eig_solver 3) only the leading eigenvalues it computed are given (every
 * selected one and at least one at or below 1/tau, unless all were
 * computed); the rest are NaN.  *count receives |Omega_Ii|. */
amdd_status amdd_get_eigenvalues(const amdd_handle* h, int32_t i, double* lam, int32_t cap,
                                 int32_t* count);

/* The |Omega_i| singular values of X_i (Eq. (Xi)) of subdomain i, descending,
 * into the host array sigma[cap]; *count receives |Omega_i|. */
amdd_status amdd_get_singular_values(const amdd_handle* h, int32_t i, double* sigma, int32_t cap,
                                     int32_t* count);

/* The coarse block of subdomain i restricted to Omega_Ii (D_i Z_i on its
 * support) as a host row-major p x nI array: p rows spanning the selected
 * eigenvectors of eq. (Zi), entries in ascending global order of Omega_Ii.
 * When the selection is partial the rows are the eigenvectors, A_II-
 * orthonormal, by descending lambda; when every eigenvalue is selected the span is all of
 * R^nI and the rows are those of diag(A_II)^{-1/2} (so E keeps the sparsity
 * of A there), or, on a handle set up with keep_coarse_matrix = 1, those of
 * L_A^{-1} (A_II = L_A L_A^T; A_II-orthonormal).  Needs cap >= p*nI. */
amdd_status amdd_get_coarse_block(const amdd_handle* h, int32_t i, double* Zt, int64_t cap,
                                  int32_t* p, int32_t* nI);

/* Kernel-class profile of a handle created with opts.profile = 1: for class
 * k in [0, AMDD_PROF_CLASSES) (one class per kernel; the two Jacobi solvers
 * are separate classes), its static name, number of launches, summed device
 * time in ms (CUDA events recorded around each launch on the stream it
 * runs on), and the algorithmic FP64 flops and DRAM bytes of those launches
 * (flops from the operation counts of the launched work; bytes for the
 * bandwidth-bound classes, 0 where not meaningful).  Counts accumulate over
 * amdd_setup, amdd_apply and amdd_pcg_solve until amdd_reset_profile.
 * Synchronises the handle's stream.  AMDD_ERR_INVALID if profiling is off or
 * k is out of range. */
#define AMDD_PROF_CLASSES 27
amdd_status amdd_get_profile(amdd_handle* h, int32_t k, const char** name, int64_t* launches, double* ms,
                             double* flops, double* bytes);

/* Clear the accumulated profile (keeps profiling on). */
amdd_status amdd_reset_profile(amdd_handle* h);

/* Largest n accepted by amdd_true_residual_noalloc. */
#define AMDD_NOALLOC_MAX_N 524288

/* No counterpart in the paper: a utility for callers that cannot allocate
 * device memory, e.g. code that runs where a framework owns every allocation
 * or a real-time loop that must not reach the allocator.  Computes the true
 * residual of a solution: out[0] = ||b - A x||_2 and out[1] = ||b||_2 (HOST
 * array of 2 doubles), with the same kernels and the same fixed reduction
 * order as the exit check of amdd_pcg_solve (stats.true_rel_residual equals
 * out[0] / out[1] for the same A, b, x).  A (device CSR), b and x (device,
 * length n) are the caller's.  It allocates nothing: its scratch is a static
 * device array of 2 * AMDD_NOALLOC_MAX_N + 272 doubles (about 8 MB) that
 * every GPU which loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (make that first call
 * before any stream capture).  Every call shares the array, so calls that
 * overlap on the GPU (other streams, other host threads) race; serialise
 * them.  AMDD_ERR_INVALID if n > AMDD_NOALLOC_MAX_N or an argument is
 * missing; work is issued on `stream` and completed before return. */
amdd_status amdd_true_residual_noalloc(const amdd_csr* A, const double* b, const double* x, double* out,
                                       void* stream);

/* Release every resource of the handle (NULL is a no-op). */
void amdd_destroy(amdd_handle* h);

/* Static description of a status code. */
const char* amdd_status_str(amdd_status s);

#ifdef __cplusplus
}
#endif

#endif /* AMDD_H */
