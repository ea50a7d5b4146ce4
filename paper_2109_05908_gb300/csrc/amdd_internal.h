// Internal declarations shared by the translation units of libamdd.
// Dense matrices are row-major: element (r, c) of a matrix with leading
// dimension ld sits at p[r * ld + c].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace amdd {

// Bits of the device error word.
enum : int {
    DERR_NOT_SPD = 1,        // Cholesky pivot <= 0 (or NaN) without clamping
    DERR_EIG_NOCONV = 2,     // Jacobi sweep limit reached
    DERR_BOUNDS = 4,         // an index check failed
    DERR_TIMEOUT = 8,        // a bounded device wait (mbarrier) gave up
};

constexpr int CHOL_NB = 32;     // diagonal block of the blocked Cholesky / inverse
constexpr int GEMM_T = 64;      // GEMM output tile
constexpr int PANEL_ROWS = 16;  // rows per CTA of the Cholesky panel solve
constexpr int GEMV_ROWS_PER_WARP = 4;  // rows per warp of the local triangular products
constexpr int MAXB = 8;                // right-hand sides per batched apply / PCG pass
constexpr int JAC_CLUSTER = 8;  // CTAs per matrix in the Jacobi solvers
constexpr int JAC_MAX_PAIRS = 64;  // largest sub-round of the shared-memory block Jacobi

// ---------------------------------------------------------------- dense
// C = alpha * op(A) * op(B) + beta * C for m x n outputs, inner dimension k.
// ta = 0: A is m x k (A[r*lda + kk]); ta = 1: A is stored k x m (A[kk*lda + r]).
// tb = 0: B is k x n (B[kk*ldb + c]); tb = 1: B is stored n x k (B[c*ldb + kk]).
// lower = 1: only elements with r >= c are written (tiles above skipped).
// kfrom_row = 1: the k loop starts at the tile's first row (for products whose
// A operand is zero for kk < r, e.g. a lower-triangular Y read transposed).
// beta == 0 means C is not read.
template <typename T>
struct GemmDescT {
    const T* A;
    const T* B;
    T* C;
    int m, n, k;
    int lda, ldb, ldc;
    int ta, tb, lower, kfrom_row;
    T alpha, beta;
};
using GemmDesc = GemmDescT<double>;

struct TileRef {
    int desc, tm, tn;
};

// Blocked Cholesky / inverse-factor descriptors (one per matrix).
template <typename T>
struct CholDescT {
    T* A;            // n x n, lower triangle used and overwritten with L
    int n, ld;
    int stop;        // factor columns [0, stop); stop < n leaves the Schur complement
    const T* clamp;  // per-matrix pivot floor (pivots below are raised to it); NULL = SPD check
    T* Linv;         // ceil(stop/NB) * NB*NB entries: inverses of the diagonal blocks
    int* bad = nullptr;  // with clamp: set to 1 when a computed pivot falls below 0.9 x the floor
                         // (or is not finite): the matrix is not numerically definite at that floor
};
using CholDesc = CholDescT<double>;

struct PanelRef {
    int desc, rt;  // row tile index (PANEL_ROWS rows) below the diagonal block
};

template <typename T>
struct TrtriDescT {
    const T* L;     // n x n lower Cholesky factor (ld)
    T* Y;           // n x n output L^{-1} (ldy), lower triangular
    const T* Linv;  // diagonal-block inverses from the Cholesky
    int n, ld, ldy;
};
using TrtriDesc = TrtriDescT<double>;

struct ChunkRef {
    int desc, ct;  // column chunk (64 columns)
};

template <typename T>
struct JacobiDescT {
    T* A;               // rows x ld, rows orthogonalised in place
    int rows, ld;
    int ncols_dot;      // columns entering the inner products
    int ncols_rot;      // columns rotated (>= ncols_dot)
    T* nrm2;            // rows scratch entries (squared row norms)
    const T* absfloor;  // optional absolute floor on |<p,q>| below which no rotation is made
};
using JacobiDesc = JacobiDescT<double>;

// Conversion descriptors of the FP32 preconditioning stage of the Jacobi solvers.
struct CvtDesc {
    const double* A;  // rows x L (lda)
    int rows, L, lda;
    float* out32;     // rows x (L + rows)
    double* Q;        // rows x rows
};

// Symmetric tridiagonal reduction and bisection (eigenvalues only).
template <typename T>
struct TridiagDescT {
    T* A;  // n x n symmetric, full storage (ld); destroyed
    int n, ld;
    T* d;  // n
    T* e;  // n (e[i] = T[i][i-1], e[0] = 0)
    T* p;  // n scratch
};
using TridiagDesc = TridiagDescT<double>;

// Row GEMV descriptors: y[row] = (b ? b[row] : 0) + alpha * sum_{c in [c0(row), c1(row))} M[row][c] x[c].
// mode 0: full row [0, ncols); mode 1: lower [0, row]; mode 2: upper [row, ncols).
template <typename T>
struct GemvDescT {
    const T* M;
    int rows, ncols, ld, mode;
    const T* x;
    T* y;
    const T* b = nullptr;  // y[row] = b[row] + alpha * (M x)[row] when b is given
    T alpha = T(1);
    const int* cstart = nullptr;  // optional per-row first column (absolute, minus coff)
    const int* cend = nullptr;    // optional per-row end column (absolute, minus coff)
    int coff = 0;
};
using GemvDesc = GemvDescT<double>;

template <typename T>
void launch_gemm(const GemmDescT<T>* d_descs, const TileRef* d_tiles, int ntiles, int tile, cudaStream_t s);
template <typename T>
void launch_chol_diag(const CholDescT<T>* d, int nmat, int k0, int* err, cudaStream_t s);
template <typename T>
void launch_chol_panel(const CholDescT<T>* d, const PanelRef* tiles, int ntiles, int k0, cudaStream_t s);
template <typename T>
void launch_trtri_diag(const TrtriDescT<T>* d, const ChunkRef* tiles, int ntiles, int k0, cudaStream_t s);
template <typename T>
void launch_set_identity(const TrtriDescT<T>* d, int nmat, int maxn, cudaStream_t s);
// Block-pair variant for matrices of any size (rows in global memory): one
// round of the block round-robin schedule (blocks of 32 rows; tasks[t] =
// {matrix, pair index in the round, blocks of that matrix (even, >= 2), 0});
// rotated[matrix] is set when a pair of it was rotated, rots[matrix] counts
// plane rotations, stats[6] accumulates pair tasks, rotated pairs, the SM
// cycles of the three phases (Gram matrix, small eigensolve, rotation of the
// rows) and the inner sweeps.  The host runs the rounds of a sweep and the sweeps.
constexpr int JP_ROWS = 32;
template <typename T>
size_t jacobi_pair_smem();
template <typename T>
void launch_jacobi_pair_round(const JacobiDescT<T>* d, const int4* tasks, int ntasks, int round, T tol, int inner,
                              int* rotated, unsigned long long* rots, unsigned long long* stats, cudaStream_t s);
// Batched FP32 GEMM on the tensor cores (tcgen05, TF32 with the 3xTF32 split
// for FP32 accuracy), 128 x 128 output tiles (TileRef tm, tn in units of 128);
// a wait that gives up latches DERR_TIMEOUT in *err.
constexpr int TC_GEMM_TILE = 128;
size_t gemm_tc_smem();
// one sweep of the block-pair Jacobi in FP32 with the Gram matrices and the
// rotations on the tensor cores (3xTF32), as one persistent launch: tasks[t] =
// {matrix, pair index in its round, blocks of that matrix, round}, ordered by
// round; CTAs claim tasks through *counter (zero before the launch) and wait
// (bounded) until bdone[bofs[matrix] + block] (zero before the launch) shows
// that both row blocks of the pair have finished the previous round; results
// are those of the round-by-round launches.  DERR_TIMEOUT into *err when a
// wait gives up.  Returns the CTAs launched.
size_t jacobi_pair_tc_smem();
int launch_jacobi_pair_tc_sweep(const JacobiDescT<float>* d, const int4* tasks, int ntasks, int* counter, int* bdone,
                                 const int* bofs, float tol, int inner, int* rotated, unsigned long long* rots,
                                 unsigned long long* stats, int* err, cudaStream_t s);
// one thread waits (bounded, `limit` SM cycles) for *flag >= 1; DERR_TIMEOUT
// into *err when the wait gives up
void launch_wait_selftest(const int* flag, long long limit, int* err, cudaStream_t s);
void launch_gemm_tc(const GemmDescT<float>* d_descs, const TileRef* d_tiles, int ntiles, int* err, cudaStream_t s);
// *p |= bits (one thread)
void launch_or_flag(int* p, int bits, cudaStream_t s);
// Shared-memory-resident block variant; returns false (nothing launched) when
// the two row blocks of the largest matrix do not fit in shared memory.
constexpr size_t JAC_BLOCK_SMEM_MAX = 220 * 1024;
template <typename T>
size_t jacobi_block_smem(int rows, int ncols_rot, int cluster);
// Shared-memory-resident block variant with a cluster of JAC_CLUSTER CTAs per
// matrix, else (blocks too large) 2 * JAC_CLUSTER; returns false, with nothing
// launched, when neither fits (smem8 / smem16: bytes per CTA for the two sizes).
template <typename T>
bool launch_jacobi_block(const JacobiDescT<T>* d, int nmat, size_t smem8, size_t smem16, int max_rows,
                         int max_sweeps, T tol, int* sweeps, unsigned long long* rots, int* err, int report_noconv,
                         cudaStream_t s);
template <typename T>
void launch_row_maxnorm2(const JacobiDescT<T>* d, int nmat, T eps, T* out, cudaStream_t s);
void launch_to_f32_with_identity(const CvtDesc* d, int nmat, int maxrows, cudaStream_t s);
void launch_extract_q(const CvtDesc* d, int nmat, int maxrows, cudaStream_t s);
// sigma[j] = ||row j|| over ncols_dot (as double); delta[mat] = eps * max_j sigma[j];
// optionally scale row j by 1/sqrt(sigma[j]).
// Robust Schur complement of the splitting (fallback when the clamped
// Cholesky of its [G, D] block is flagged): rows of C = Sigma^{1/2} V^T
// (n_i x nt, columns [C_R | C_I], C_R the first nR) give
//   J = [C_R | I_{n_i}]  (n_i x (nR + n_i), leading dimension ldj), and after
//   the one-sided Jacobi of J's rows (inner products over the first nR
//   columns) each row k of its right part is scaled by 1 / sqrt(s_k^2 + delta)
//   with s_k^2 the squared norm of its left part.
template <typename T>
struct KjacDesc {
    const T* C;  // n_i x nt (ldc)
    T* J;        // n_i x (nR + n_i) (ldj)
    int ni, nR, ldc, ldj;
    const T* delta;
};
// Coarse block of a subdomain whose every eigenvalue is selected: the nI x nI
// rows Zt[k][c] = (k == c) / sqrt(A_II[k][k]) (A_ii dense FP64, leading
// dimension lda).
struct DiagBasisDesc {
    const double* A;
    int lda;
    double* Zt;
    int nI;
};
void launch_diag_basis(const DiagBasisDesc* d, int nmat, int maxn, cudaStream_t s);
// With that basis: AZ[r][c] = A_ii[r][c] / sqrt(A_II[c][c]) (ni x nI, leading
// dimension nI) and the lower triangle of E_ii[r][c] = AZ[r][c] / sqrt(A_II[r][r])
// (leading dimension ldE).
struct DiagScaleDesc {
    const double* A;  // A_ii dense, ni x ni (leading dimension ni)
    int ni, nI;
    double* AZ;
    double* Eii;
    int64_t ldE;
};
void launch_diag_scale(const DiagScaleDesc* d, int nmat, int maxni, cudaStream_t s);
// Matrix-free local eigensolve (eq. (invAii)): from the scaled rows C =
// Sigma^{1/2} V^T of the SVD of X_i (ni x nt, leading dimension ld, the
// Omega_Ii columns from nR on) and the row norms sigma, Cc = C(:, I) and
// Bm = diag(1 / (sigma + delta)) C(:, I), both ni x nI contiguous.
struct MfPrepDesc {
    const double* X1;
    int ld, nR, ni, nI;
    const double* sig;    // sigma_j of row j
    const double* delta;  // sigma_1 eps (one value)
    double* Cc;
    double* Bm;
};
void launch_mf_prepare(const MfPrepDesc* d, int nmat, int maxni, cudaStream_t s);
template <typename T>
void launch_build_kjac(const KjacDesc<T>* d, int nmat, int maxrows, cudaStream_t s);
template <typename T>
void launch_kjac_scale(const KjacDesc<T>* d, int nmat, cudaStream_t s);
template <typename T>
void launch_rownorms(const JacobiDescT<T>* d, int nmat, double* const* sigma_ptrs, T* delta, double eps,
                     int scale_rows, cudaStream_t s);
template <typename T>
void launch_add_diag(T* const* mats, const int* n, const int* ld, const T* delta, int nmat, int maxn, cudaStream_t s);
template <typename T>
void launch_mirror_lower(T* const* mats, const int* n, const int* ld, int nmat, int maxn, cudaStream_t s);
template <typename T>
void launch_transpose(const T* const* src, T* const* dst, const int* n, const int* lds, const int* ldd, int nmat,
                      int maxn, cudaStream_t s);
template <typename T>
void launch_gemv_rows(const GemvDescT<T>* d, const int* row_desc, const int* row_local, int64_t nrows,
                      cudaStream_t s);
template <typename T>
void launch_gemv_rows4(const GemvDescT<T>* d, const int* grp_desc, const int* grp_row, int64_t ngroups,
                       cudaStream_t s);
template <typename T>
void launch_gemv_rows4_multi(const GemvDescT<T>* d, const int* grp_desc, const int* grp_row, int64_t ngroups, int nb,
                             int64_t xs, int64_t ys, cudaStream_t s);
template <typename T>
void launch_gemv_rows_multi(const GemvDescT<T>* d, const int* row_desc, const int* row_local, int64_t nrows, int nb,
                            int64_t xs, int64_t ys, cudaStream_t s);
template <typename T>
void launch_tridiag(const TridiagDescT<T>* d, int nmat, int maxn, cudaStream_t s);
template <typename T>
void launch_bisect(const TridiagDescT<T>* d, int nmat, const int* eig_mat, const int* eig_idx, int64_t total,
                   double* const* out, cudaStream_t s);
// dst[i] = (To)src[i]
template <typename Ti, typename To>
void launch_convert(const Ti* src, To* dst, int64_t n, cudaStream_t s);
template <typename Ti, typename To>
void launch_convert_blocks(const Ti* const* src, const int* lds, To* const* dst, const int* ldd, const int* n,
                           int nmat, int maxn, cudaStream_t s);

// ---------------------------------------------------------------- sparse / vectors
// Sparse local Cholesky factors: per subdomain its order n, factor entries
// nnz, the offset of its column pointers (n + 1 local offsets), of its entries
// and of its rows in the local vectors.
struct SparseLocalDesc {
    int n, nnz;
    int64_t poff, eoff, xoff;
};
// dst[t] = src[idx[t]] (idx >= 0) or 1 / src[-idx[t] - 1]
template <typename T>
void launch_gather_entries(const T* src, const int64_t* idx, T* dst, int64_t cnt, cudaStream_t s);
// y_i = P^T L^{-T} L^{-1} P r_i with the factors staged in shared memory (smem:
// the largest sparse_local_smem of the batch for nb vectors), nb <= MAXB
// vectors ld apart
template <typename T>
size_t sparse_local_smem(int n, int nnz, int nb);
template <typename T>
void launch_sparse_local_solve(const SparseLocalDesc* d, int nmat, size_t smem, const int32_t* colptr,
                               const uint16_t* rowidx, const T* val, const int32_t* perm, const T* r, T* y, int nb,
                               int64_t ld, cudaStream_t s);

// Host: nested-dissection order of the symmetric pattern of an n x n CSR graph
// (sets of at most `leaf` unknowns not cut) and the column structure of the
// Cholesky factor of P A P^T in that order: perm[k] = old index of new k,
// column j holds rows[colptr[j] .. colptr[j+1]), the diagonal j first, then
// ascending.  False on a malformed graph.
bool nd_factor_pattern(int n, const int64_t* rowptr, const int32_t* colind, int leaf, std::vector<int32_t>& perm,
                       std::vector<int32_t>& colptr, std::vector<int32_t>& rows);

// *flag |= 1 when v[0..n) holds a NaN or an infinity
void launch_nonfinite(const double* v, int64_t n, int* flag, cudaStream_t s);
// Lanes per row of launch_spmv for a matrix of n rows and nnz entries: the one
// choice every SpMV of the library makes, so that equal inputs give equal bits
int spmv_group_for(int64_t n, int64_t nnz);
void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y, int group, cudaStream_t s);
void launch_gather_values(const int64_t* src, const int64_t* dst, int64_t cnt, const double* val, double* out,
                          cudaStream_t s);
void launch_gather_vec(const int32_t* idx, int64_t cnt, const double* x, double* out, cudaStream_t s);
void launch_gather_vec_multi(const int32_t* idx, int64_t cnt, const double* x, int64_t ldx, double* out, int nb,
                             cudaStream_t s);
void launch_spmv_multi(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                       double* y, int nb, int64_t ld, cudaStream_t s);
template <typename T>
void launch_gather_rows(const T* src, const int64_t* src_off, T* dst, const int64_t* dst_off, const int32_t* len,
                        int64_t nrows, cudaStream_t s);
template <typename TY>
void launch_scatter_prolong(int64_t n, const int32_t* order_g, const int64_t* sc_ptr, const int32_t* sc_idx,
                            const TY* yloc, const double* zc, double* z, cudaStream_t s, int nb = 1, int64_t ldy = 0,
                            int64_t ldzc = 0, int64_t ldz = 0);
// batched rectangular transposes: dst (cols x rows, leading dimension ldd) = src^T
struct TransDesc {
    const double* src;
    double* dst;
    int rows, cols, lds, ldd;
};
void launch_transpose_rect(const TransDesc* d, int nmat, int maxdim, cudaStream_t s);
struct EPairRef {
    int i, j;          // block E_ij, i > j
    int64_t list_off;  // entries [list_off, list_off + list_len)
    int list_len;
    int tr, tc;        // 32x32 tile of the p_i x p_j block
};
void launch_e_offdiag(const EPairRef* tiles, int ntiles, const int32_t* la, const int32_t* lpos,
                      const double* Zt, const int64_t* zt_off, const int32_t* nI, const double* AZ,
                      const int64_t* az_off, const int32_t* p, const int64_t* coff, double* E, int64_t ldE,
                      cudaStream_t s);

// Deterministic dot products: fixed grid of DOT_BLOCKS partial sums reduced in
// a fixed order by one block.
constexpr int DOT_BLOCKS = 264;
// ---------------------------------------------------------------------------
// Learned warm start of the local eigensolve and block LOBPCG
// ---------------------------------------------------------------------------
constexpr int PROP_NF = 32;    // features per subdomain
constexpr int PROP_NB = 16;    // Krylov basis vectors
constexpr int PROP_NH = 256;   // hidden width
constexpr int PROP_NO = 256;   // outputs: a 16 x 16 matrix
// parameter layout: W1 (32 x 256), b1, W2 (256 x 256), b2, W3 (256 x 256), b3
constexpr int64_t MLP_OFF_W1 = 0;
constexpr int64_t MLP_OFF_B1 = MLP_OFF_W1 + PROP_NF * PROP_NH;
constexpr int64_t MLP_OFF_W2 = MLP_OFF_B1 + PROP_NH;
constexpr int64_t MLP_OFF_B2 = MLP_OFF_W2 + PROP_NH * PROP_NH;
constexpr int64_t MLP_OFF_W3 = MLP_OFF_B2 + PROP_NH;
constexpr int64_t MLP_OFF_B3 = MLP_OFF_W3 + PROP_NH * PROP_NO;
constexpr int64_t MLP_NPARAM = MLP_OFF_B3 + PROP_NO;

// Features of subdomain i from its dense local matrix A_ii (rows [I, G],
// leading dimension ld, ncols = |Omega_i|):
//  0 log nI, 1 log(1+nG), 2 log(1+nD), 3 nG/nI, 4 nD/nI,
//  5-8 mean/std/min/max of log diag(A_II), 9-12 the same of log|off-diagonal
//  non-zeros of A_II|, 13 max - min of log diag, 14-16 mean/std/max of the
//  off-diagonal non-zeros per row, 17 fraction of rows coupled to Omega_G,
//  18-19 mean/max of sum_G |a_rg| / a_rr, 20-23 mean/std/min/max of
//  sum_{c != r} |a_rc| / a_rr, 24 log(||A_II||_F / nI), 25 log(trace / nI),
//  26 fraction of positive off-diagonal non-zeros, 27 log(max(p,1)/nI),
//  28 log max(p,1), 29 log tau, 30 mean log diag over coupled rows minus
//  the mean over all rows, 31 the constant 1.
struct FeatDesc {
    const double* A;
    int ld, ncols, nI, nG, nD, p;
    double tau;
    float* out;  // 32 entries
};
void launch_features(const FeatDesc* d, int nmat, cudaStream_t s);

struct KrylovDesc {
    const double* A;  // A_II is the leading nI x nI block (leading dimension ld)
    int ld, nI;
    double* Bt;  // PROP_NB x nI, rows = basis vectors
    double* w;   // nI scratch
};
void launch_krylov(const KrylovDesc* d, int nmat, cudaStream_t s);

// mean[f], sd[f] (population; < 1e-6 -> 1) of the columns of an n x PROP_NF matrix
void launch_feature_stats(const float* feat, int n, float* mean, float* sd, cudaStream_t s);
void launch_normalize_features(const float* feat, const float* mean, const float* sd, float* X, int n,
                               cudaStream_t s);
void launch_bias_act(float* Z, const float* bias, float* H, int rows, int cols, cudaStream_t s);
void launch_symmetrise(const float* Y, float* Q, int n, cudaStream_t s);
void launch_loss_grad(const float* Q, const float* Qt, float* dY, float* part, float* loss, int n, cudaStream_t s);
void launch_relu_back(const float* dH, const float* Z, float* dZ, int n, cudaStream_t s);
void launch_colsum(const float* dZ, float* db, int rows, int cols, cudaStream_t s);
void launch_adam(float* W, float* Wb, float* m, float* v, const float* g, int n, float lr, int t, cudaStream_t s);
void launch_bf16_round(const float* W, float* Wb, int n, cudaStream_t s);

template <typename T>
struct RowsDesc {  // rows [r0, r1) of a row-major matrix (cols entries each)
    T* A;
    int ld, r0, r1, cols, id;
};
template <typename T>
void launch_rng_rows(const RowsDesc<T>* d, int nmat, int maxrows, unsigned long long seed, cudaStream_t s);

template <typename T>
void launch_zero_upper(const RowsDesc<T>* d, int nmat, int maxrows, cudaStream_t s);
// out[t] = dot of the two halves (len[t] entries each) of the row at W + off[t]
template <typename T>
void launch_half_dots(const T* W, const int64_t* off, const int32_t* len, int64_t rows, double* out, cudaStream_t s);

template <typename T>
struct ResidDesc {  // R = TX - diag(theta) X over k rows of n entries; norms of the first `want`
    const T* X;
    const T* TX;
    T* R;
    const T* theta;
    double* norms;
    int ld, n, k, want;
};
template <typename T>
void launch_residual_rows(const ResidDesc<T>* d, int nmat, cudaStream_t s);

template <typename T>
struct ScaleDesc {  // A[r] *= f[r] (or 1 / ||A[r]|| with unit scaling)
    T* A;
    int ld, rows, cols;
    const T* f;
};
template <typename T>
void launch_scale_rows(const ScaleDesc<T>* d, int nmat, int unit, cudaStream_t s);

// Coarse solve L_E L_E^T e = c (one cooperative launch; c is overwritten).
struct CoarseSolveArgs {
    const double* L;       // factor, n x n row-major (lower), leading dimension ld
    const double* Lt;      // its transpose, row-major
    const double* Yd;      // K inverses of the SB x SB diagonal blocks (lower), SB x SB each
    const double* Ydt;     // their transposes
    const int* env_row;    // first non-zero column of row r of L
    const int* env_colend; // one past the last non-zero row of column r of L
    double* c;             // right-hand side, overwritten
    double* y;             // work (n)
    double* e;             // solution (n)
    int n, ld, SB, K;
    int nb = 1;            // right-hand sides (c, y, e hold nb vectors ldv apart)
    int64_t ldv = 0;
    // Folded form (F != NULL), one grid-wide phase per block and direction:
    //   y_k = Yd_k c_k - F_k y[fw0_k, r0_k),   F_k = Yd_k L(block k, [fw0_k, r0_k))
    //   e_k = Ydt_k y_k - G_k e[r1_k, gw1_k),  G_k = Ydt_k L^T(block k, [r1_k, gw1_k))
    // F_k and G_k are SB x FW row-major blocks (K of each); c is not overwritten.
    const double* F = nullptr;
    const double* G = nullptr;
    const int* fw0 = nullptr;
    const int* gw1 = nullptr;
    int FW = 0;
};
int coarse_solve_blocks();  // cooperative grid size for this device (0 on error)
cudaError_t launch_coarse_solve(const CoarseSolveArgs& a, int blocks, cudaStream_t s);

struct PcgScal {
    double rz, pq, rr, bb, alpha, beta, rz_new;
    int conv, iters;
};
// Vector operations of PCG on nb right-hand sides stored ld apart (scalars sc[k],
// partial sums DOT_BLOCKS apart); with skip_done a converged right-hand side
// (sc[k].conv) keeps x, r, p and its scalars.
void launch_dot_partials(int64_t n, const double* x, const double* y, double* partials, cudaStream_t s, int nb = 1,
                         int64_t ld = 0);
// which: 0 -> pq (alpha = rz/pq), 1 -> rz_new (beta = rz_new/rz, rz = rz_new),
// 2 -> rr (conv = rr <= tol2 * bb), 3 -> bb, 4 -> rz (initial)
void launch_dot_finalize(const double* partials, PcgScal* sc, int which, double tol2, cudaStream_t s, int nb = 1,
                         int skip_done = 0);
void launch_pcg_update_xr(int64_t n, double* x, double* r, const double* p, const double* q, const PcgScal* sc,
                          double* partials, cudaStream_t s, int nb = 1, int64_t ld = 0, int skip_done = 0);
void launch_pcg_update_p(int64_t n, double* p, const double* z, const PcgScal* sc, cudaStream_t s, int nb = 1,
                         int64_t ld = 0, int skip_done = 0);
void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);
// One thread: alog[k-1] = sc->alpha, blog[k-2] = sc->beta (k = sc->iters, entries
// below *maxit only), then the while-loop condition of the graph that replays
// PCG iterations: !sc->conv && k < *maxit.
void launch_pcg_loop_cond(const PcgScal* sc, const int* maxit, double* alog, double* blog,
                          cudaGraphConditionalHandle loop, cudaStream_t s);

// ---------------------------------------------------------------------------
// Deflated / restricted additive Schwarz forms and GMRES(m) (Sec. 4.1)
// ---------------------------------------------------------------------------
// z[order_g[t]] = yloc[own_idx[t]] (+ zc[t] when zc is given)
template <typename TY>
void launch_ras_prolong(int64_t n, const int32_t* order_g, const int32_t* own_idx, const TY* yloc, const double* zc,
                        double* z, cudaStream_t s);
// zg[order_g[t]] = zo[t]
void launch_owner_to_global(int64_t n, const int32_t* order_g, const double* zo, double* zg, cudaStream_t s);
// Ep[r][c] = E[perm r][perm c] for c <= r (E and Ep lower triangles of n x n
// row-major matrices; Ep's upper triangle is zeroed)
void launch_sym_permute(const double* E, double* Ep, const int32_t* perm, int64_t n, cudaStream_t s);
// dst[k*ld + r] = src[k*ld + perm[r]] / dst[k*ld + perm[r]] = src[k*ld + r], r < n, k < nb
void launch_perm_gather(int64_t n, const int32_t* perm, const double* src, double* dst, int nb, int64_t ld,
                        cudaStream_t s);
void launch_perm_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, int nb, int64_t ld,
                         cudaStream_t s);
// out[t] = val[src[t]] (64-bit indices)
void launch_gather_idx64(const int64_t* src, int64_t cnt, const double* val, double* out, cudaStream_t s);
// y = b - A x
void launch_spmv_resid(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                       const double* b, double* y, int group, cudaStream_t s);

constexpr int GM_MAXR = 64;   // largest GMRES restart length
constexpr int GM_CHUNK = 32;  // basis vectors per block row of the fused Gram-Schmidt passes
struct GmState {
    double H[GM_MAXR * (GM_MAXR + 1)];  // Hessenberg matrix, column-major (column j: rows 0..j+1), rotated
    double cs[GM_MAXR], sn[GM_MAXR];    // Givens rotations
    double g[GM_MAXR + 1];              // rotated right-hand side beta e_1
    double y[GM_MAXR];                  // least-squares solution of a cycle
    double hcol[GM_MAXR + 1];           // projections of the current Gram-Schmidt pass
    double bnorm2, beta, hnext, res;    // ||b||^2, ||r_0|| of the cycle, h_{j+1,j}, |g_{j+1}| / ||b||
    int conv;
};
void launch_gm_ortho(int64_t n, const double* V, int64_t ldv, int k, const double* h, const double* w, double* out,
                     double* part, int mode, cudaStream_t s);
void launch_gm_finalize(const double* part, int k, double* hcol, double* Hcol, int add, cudaStream_t s);
void launch_gm_norm(const double* part, GmState* st, int which, cudaStream_t s);
void launch_gm_givens(const double* part, GmState* st, int j, double rtol, cudaStream_t s);
void launch_gm_scale(int64_t n, const double* src, double* dst, const GmState* st, int which, cudaStream_t s);
void launch_gm_trisolve(GmState* st, int k, cudaStream_t s);
void launch_gm_combine(int64_t n, const double* Zp, int64_t ldv, int k, const GmState* st, double* x,
                       cudaStream_t s);

}  // namespace amdd
