// Batched dense kernels (FP64, and FP32 for the mixed-precision form) for the
// subdomain blocks of the setup:
// tiled GEMM, blocked Cholesky (full or stopped early to leave a Schur
// complement), blocked inverse of the Cholesky factor, one-sided Jacobi row
// orthogonalisation (SVD of X_i, Sec. 3.2, and the symmetric eigensolve of
// eq. (Zi)), and small helpers.  One launch serves every subdomain at once
// (uneven sizes through per-matrix descriptors and flat tile lists).
#include <cooperative_groups.h>

#include "amdd_internal.h"
#include "jacobi_pair_inner.cuh"

#include <limits>

namespace cg = cooperative_groups;

namespace amdd {

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// ------------------------------------------------------------------ GEMM
// TILE x TILE output tile per CTA, RM x 4 outputs per thread (threads =
// TILE/RM x TILE/4), k staged through shared memory 16 at a time, FMA in the
// element type.  TILE = 64 (4 x 4 per thread, 256 threads) for wide batches;
// TILE = 32 (2 x 4 per thread, 128 threads) gives four times as many CTAs
// when one launch would not fill the SMs (the coarse factorisation), with
// four warps per CTA so each SM sub-partition has one to issue from.
constexpr int GK = 16;

template <typename T, int TILE, int RM>
__global__ void __launch_bounds__((TILE / RM) * (TILE / 4)) gemm_tiles_kernel(const GemmDescT<T>* __restrict__ descs,
                                                                              const TileRef* __restrict__ tiles,
                                                                              int ntiles) {
    constexpr int TX = TILE / 4;   // threads along a tile row (4 columns each)
    constexpr int TY = TILE / RM;  // threads along a tile column (RM rows each)
    constexpr int NT = TX * TY;
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const TileRef tr = tiles[t];
    const GemmDescT<T> d = descs[tr.desc];
    __shared__ T As[GK][TILE + 1];
    __shared__ T Bs[GK][TILE + 1];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int row0 = tr.tm * TILE, col0 = tr.tn * TILE;
    T acc[RM][4];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    int kbeg = 0;
    if (d.kfrom_row) kbeg = (row0 / GK) * GK;
    for (int k0 = kbeg; k0 < d.k; k0 += GK) {
        for (int e = tid; e < TILE * GK; e += NT) {
            int r, kk;
            if (!d.ta) { r = e / GK; kk = e % GK; } else { kk = e / TILE; r = e % TILE; }
            const int gr = row0 + r, gk = k0 + kk;
            T v = T(0);
            if (gr < d.m && gk < d.k)
                v = d.ta ? d.A[(size_t)gk * d.lda + gr] : d.A[(size_t)gr * d.lda + gk];
            As[kk][r] = v;
        }
        for (int e = tid; e < TILE * GK; e += NT) {
            int c, kk;
            if (!d.tb) { kk = e / TILE; c = e % TILE; } else { c = e / GK; kk = e % GK; }
            const int gc = col0 + c, gk = k0 + kk;
            T v = T(0);
            if (gc < d.n && gk < d.k)
                v = d.tb ? d.B[(size_t)gc * d.ldb + gk] : d.B[(size_t)gk * d.ldb + gc];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            T a[RM], b[4];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int r = row0 + ty + TY * i;
        if (r >= d.m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx + TX * j;
            if (c >= d.n || (d.lower && c > r)) continue;
            T* cp = d.C + (size_t)r * d.ldc + c;
            const T v = d.alpha * acc[i][j];
            *cp = (d.beta != T(0)) ? fma(d.beta, *cp, v) : v;
        }
    }
}

template <typename T>
void launch_gemm(const GemmDescT<T>* d_descs, const TileRef* d_tiles, int ntiles, int tile, cudaStream_t s) {
    if (ntiles <= 0) return;
    if (tile == 16)
        gemm_tiles_kernel<T, 16, 1><<<ntiles, 64, 0, s>>>(d_descs, d_tiles, ntiles);
    else if (tile == 32)
        gemm_tiles_kernel<T, 32, 2><<<ntiles, 128, 0, s>>>(d_descs, d_tiles, ntiles);
    else
        gemm_tiles_kernel<T, 64, 4><<<ntiles, 256, 0, s>>>(d_descs, d_tiles, ntiles);
}
template void launch_gemm<float>(const GemmDescT<float>*, const TileRef*, int, int, cudaStream_t);
template void launch_gemm<double>(const GemmDescT<double>*, const TileRef*, int, int, cudaStream_t);

// ------------------------------------------------------------------ Cholesky
// Factor the NB x NB diagonal block [k0, k0+kb) of each matrix in shared
// memory (its trailing part already updated by earlier steps), write L back
// and store the inverse of the block for the panel solve and for the inverse
// factor.  With a pivot floor (clamp) a pivot below it is raised to it;
// without, a pivot <= 0 (or NaN) latches DERR_NOT_SPD and is replaced by 1 so
// the factorisation finishes with finite numbers.
//
// Column j keeps its unscaled entries a_rj; the update of step j is
// a_rc -= a_rj a_cj / d_j over the active lower triangle j < c <= r, listed
// by a table whose active part is a prefix at every step (columns in
// descending order).  The thread that updates the next pivot also takes its
// reciprocal square root, so one barrier per column suffices.  The inverse of
// the factor is formed blockwise: four 8 x 8 diagonal inverses, then two
// levels of [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}].
constexpr int DIAG_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) chol_diag_kernel(const CholDescT<T>* __restrict__ descs, int k0,
                                                                  int* __restrict__ err) {
    const CholDescT<T> d = descs[blockIdx.x];
    const int kend = min(k0 + CHOL_NB, d.stop);
    if (k0 >= kend) return;
    const int kb = kend - k0;
    __shared__ T L[CHOL_NB][CHOL_NB + 1];   // working entries; the factor F overwrites column j after step j
    __shared__ T Li[CHOL_NB][CHOL_NB + 1];  // inverse of the factor
    __shared__ T Xs[CHOL_NB][CHOL_NB + 1];  // products of the blocked inverse
    __shared__ T piv[CHOL_NB];              // pivot d_j (after clamping)
    __shared__ T rinv[CHOL_NB];             // 1 / sqrt(d_j)
    __shared__ unsigned short tab[CHOL_NB * (CHOL_NB + 1) / 2];
    const int tid = threadIdx.x;
    const T floor_v = d.clamp ? *d.clamp : T(0);
    // padded to NB: rows / columns >= kb are the identity
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += DIAG_THREADS) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        T v = T(0);
        if (r < kb && c <= r) v = d.A[(size_t)(k0 + r) * d.ld + (k0 + c)];
        else if (r == c) v = T(1);
        L[r][c] = v;
        if (c <= r && r < kb) {
            const int q = kb - 1 - c;
            tab[q * (q + 1) / 2 + (r - c)] = (unsigned short)((r << 8) | c);
        }
    }
    __syncthreads();
    auto take_pivot = [&](int j, T a) {
        T p = a;
        if (d.clamp) {
            // exact pivots of a matrix >= floor * I are >= floor: one well below
            // it means rounding has destroyed the definiteness
            if (d.bad && !(p >= T(0.9) * floor_v && isfinite(p))) *d.bad = 1;
            if (!(p >= floor_v)) p = floor_v;
        } else if (!(p > T(0))) {
            atomicOr(err, DERR_NOT_SPD);
            p = T(1);
        }
        piv[j] = p;
        rinv[j] = rsqrt_t(p);
    };
    if (tid == 0) take_pivot(0, L[0][0]);
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        const T rj = rinv[j];
        const T s = rj * rj;
        const int m = (kb - 1 - j) * (kb - j) / 2;
        for (int e = tid; e < m; e += DIAG_THREADS) {
            const int rc = tab[e];
            const int r = rc >> 8, c = rc & 255;
            const T v = fma(-(L[r][j] * s), L[c][j], L[r][c]);
            L[r][c] = v;
            if (r == j + 1 && c == j + 1) take_pivot(j + 1, v);
        }
        __syncthreads();
        // column j of the factor (entries below the diagonal are not read again)
        if (tid < kb - j) {
            const int r = j + tid;
            L[r][j] = (r == j) ? piv[j] * rj : L[r][j] * rj;
        }
    }
    for (int r = kb + tid; r < CHOL_NB; r += DIAG_THREADS) rinv[r] = T(1);
    __syncthreads();
    // ---- inverse of the factor, blockwise
    const int warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += DIAG_THREADS) Li[e / CHOL_NB][e % CHOL_NB] = T(0);
    __syncthreads();
    if (lane < 8) {  // warp w inverts the 8 x 8 diagonal block w, one column per lane
        const int b0 = warp * 8, c = b0 + lane;
        for (int r = c; r < b0 + 8; ++r) {
            T acc = (r == c) ? T(1) : T(0);
            for (int k = c; k < r; ++k) acc = fma(-L[r][k], Li[k][c], acc);
            Li[r][c] = acc * rinv[r];
        }
    }
    __syncthreads();
    for (int w = 8; w < CHOL_NB; w *= 2) {
        // pairs of w x w diagonal blocks [A 0; B C] at offsets o = 0, 2w, ...
        const int npairs = CHOL_NB / (2 * w);
        // X = B A^{-1}  (w x w per pair)
        for (int e = tid; e < npairs * w * w; e += DIAG_THREADS) {
            const int pr = e / (w * w), rr = (e / w) % w, cc = e % w;
            const int o = pr * 2 * w;
            T acc = T(0);
            for (int k = cc; k < w; ++k) acc = fma(L[o + w + rr][o + k], Li[o + k][o + cc], acc);
            Xs[o + w + rr][o + cc] = acc;
        }
        __syncthreads();
        // lower-left block = -C^{-1} X
        for (int e = tid; e < npairs * w * w; e += DIAG_THREADS) {
            const int pr = e / (w * w), rr = (e / w) % w, cc = e % w;
            const int o = pr * 2 * w;
            T acc = T(0);
            for (int k = 0; k <= rr; ++k) acc = fma(Li[o + w + rr][o + w + k], Xs[o + w + k][o + cc], acc);
            Li[o + w + rr][o + cc] = -acc;
        }
        __syncthreads();
    }
    T* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += DIAG_THREADS) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        if (r < kb && c <= r) d.A[(size_t)(k0 + r) * d.ld + (k0 + c)] = L[r][c];
        linv[e] = (r < kb && c < kb) ? Li[r][c] : T(0);
    }
}

template <typename T>
void launch_chol_diag(const CholDescT<T>* d, int nmat, int k0, int* err, cudaStream_t s) {
    if (nmat > 0) chol_diag_kernel<T><<<nmat, DIAG_THREADS, 0, s>>>(d, k0, err);
}
template void launch_chol_diag<float>(const CholDescT<float>*, int, int, int*, cudaStream_t);
template void launch_chol_diag<double>(const CholDescT<double>*, int, int, int*, cudaStream_t);

// Panel below the diagonal block: A[r, k0:k0+kb] <- A[r, k0:k0+kb] * Linv^T
// for PANEL_ROWS rows per CTA.
template <typename T>
__global__ void __launch_bounds__(256) chol_panel_kernel(const CholDescT<T>* __restrict__ descs,
                                                          const PanelRef* __restrict__ tiles, int k0) {
    const PanelRef t = tiles[blockIdx.x];
    const CholDescT<T> d = descs[t.desc];
    const int kend = min(k0 + CHOL_NB, d.stop);
    const int kb = kend - k0;
    const int r0 = kend + t.rt * PANEL_ROWS;
    __shared__ T Li[CHOL_NB][CHOL_NB + 1];
    __shared__ T P[PANEL_ROWS][CHOL_NB + 1];
    const T* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += 256) Li[e / CHOL_NB][e % CHOL_NB] = linv[e];
    for (int e = tid; e < PANEL_ROWS * CHOL_NB; e += 256) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        const int gr = r0 + r;
        P[r][c] = (gr < d.n && c < kb) ? d.A[(size_t)gr * d.ld + (k0 + c)] : T(0);
    }
    __syncthreads();
    // lanes run over rows so the loop length (c + 1) is uniform in a warp
    for (int e = tid; e < PANEL_ROWS * CHOL_NB; e += 256) {
        const int c = e / PANEL_ROWS, r = e % PANEL_ROWS;
        const int gr = r0 + r;
        if (c < kb && gr < d.n) {
            T s = T(0);
            for (int k = 0; k <= c; ++k) s = fma(P[r][k], Li[c][k], s);
            d.A[(size_t)gr * d.ld + (k0 + c)] = s;
        }
    }
}

template <typename T>
void launch_chol_panel(const CholDescT<T>* d, const PanelRef* tiles, int ntiles, int k0, cudaStream_t s) {
    if (ntiles > 0) chol_panel_kernel<T><<<ntiles, 256, 0, s>>>(d, tiles, k0);
}
template void launch_chol_panel<float>(const CholDescT<float>*, const PanelRef*, int, int, cudaStream_t);
template void launch_chol_panel<double>(const CholDescT<double>*, const PanelRef*, int, int, cudaStream_t);

// ------------------------------------------------------------------ inverse factor
// Y = L^{-1} by blocked forward substitution on the identity: for each
// diagonal block k, Y[k-rows, 0:kend] <- Linv_k * Y[k-rows, 0:kend]; the
// trailing update Y[kend:, 0:kend] -= L[kend:, k-cols] * Y[k-rows, 0:kend]
// is a GEMM issued by the host.
template <typename T>
__global__ void __launch_bounds__(256) trtri_diag_kernel(const TrtriDescT<T>* __restrict__ descs,
                                                          const ChunkRef* __restrict__ tiles, int k0) {
    const ChunkRef t = tiles[blockIdx.x];
    const TrtriDescT<T> d = descs[t.desc];
    const int kend = min(k0 + CHOL_NB, d.n);
    const int kb = kend - k0;
    const int c0 = t.ct * 64;
    __shared__ T Li[CHOL_NB][CHOL_NB + 1];
    __shared__ T B[CHOL_NB][64 + 1];
    const T* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += 256) Li[e / CHOL_NB][e % CHOL_NB] = linv[e];
    for (int e = tid; e < CHOL_NB * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        B[r][c] = (r < kb && c0 + c < kend) ? d.Y[(size_t)(k0 + r) * d.ldy + (c0 + c)] : T(0);
    }
    __syncthreads();
    for (int e = tid; e < CHOL_NB * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        if (r < kb && c0 + c < kend) {
            T s = T(0);
            for (int k = 0; k <= r; ++k) s = fma(Li[r][k], B[k][c], s);
            d.Y[(size_t)(k0 + r) * d.ldy + (c0 + c)] = s;
        }
    }
}

template <typename T>
void launch_trtri_diag(const TrtriDescT<T>* d, const ChunkRef* tiles, int ntiles, int k0, cudaStream_t s) {
    if (ntiles > 0) trtri_diag_kernel<T><<<ntiles, 256, 0, s>>>(d, tiles, k0);
}
template void launch_trtri_diag<float>(const TrtriDescT<float>*, const ChunkRef*, int, int, cudaStream_t);
template void launch_trtri_diag<double>(const TrtriDescT<double>*, const ChunkRef*, int, int, cudaStream_t);

template <typename T>
__global__ void set_identity_kernel(const TrtriDescT<T>* __restrict__ descs) {
    const TrtriDescT<T> d = descs[blockIdx.y];
    for (int r = blockIdx.x; r < d.n; r += gridDim.x) {
        T* row = d.Y + (size_t)r * d.ldy;
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) row[c] = (r == c) ? T(1) : T(0);
    }
}

template <typename T>
void launch_set_identity(const TrtriDescT<T>* d, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid(min(maxn, 1024), nmat);
    set_identity_kernel<T><<<grid, 256, 0, s>>>(d);
}
template void launch_set_identity<float>(const TrtriDescT<float>*, int, int, cudaStream_t);
template void launch_set_identity<double>(const TrtriDescT<double>*, int, int, cudaStream_t);

// ------------------------------------------------------------------ Jacobi
// One-sided (Hestenes) Jacobi on the rows of each matrix, in T = float or
// double: rotate row pairs until every pair is orthogonal over the first
// ncols_dot columns to tol relative to the row norms (and, when a floor is
// given, above that absolute floor on |<p,q>|); rotations are applied to
// ncols_rot columns (so an identity appended on the right accumulates them).
// Two forms below: the rows resident in the shared memory of a cluster (block
// kernel) when they fit, else block pairs with the rows in global memory.
// Rotation that makes rows p, q (Gram [[a, g], [g, b]]) orthogonal:
// t = tan(theta) is the smaller root of t^2 + 2 zeta t - 1 = 0, zeta =
// (b - a) / (2 g), written as t = sign(b - a) 2 g / (|b - a| + sqrt((b - a)^2 +
// 4 g^2)) so that one square root, one division and one reciprocal square
// root suffice; cs = 1/sqrt(1 + t^2), sn = cs t.

template <typename T>
__device__ __forceinline__ void jac_rotation(T a, T b, T g, T& cs, T& sn, T& t) {
    const T dd = b - a;
    const T g2 = g + g;
    t = copysign(T(1), dd) * g2 / (fabs(dd) + sqrt(fma(dd, dd, g2 * g2)));
    cs = rsqrt_t(fma(t, t, T(1)));
    sn = cs * t;
}

// ------------------------------------------------------------------ block-pair Jacobi
// The same one-sided Jacobi for matrices whose rows do not fit in shared
// memory.  Rows are cut into blocks of JP_B; a sweep meets every two blocks
// once in a round-robin (circle) schedule, one launch per round for all
// matrices and all disjoint block pairs of the round.  For a pair (I, J) one
// CTA
//   1. forms the Gram matrix G = Y Y^T of the JP_R = 2 JP_B rows
//      Y = [Y_I; Y_J] over the first ncols_dot columns (columns streamed
//      through shared memory, 4 x 4 outputs per thread);
//   2. diagonalises G in shared memory by two-sided cyclic Jacobi with the
//      rotation, the stopping test and the absolute floor of the row kernel:
//      in exact arithmetic the two-sided rotation of G is the Gram matrix of
//      the one-sided rotation of the rows, so the composed rotation Q^T
//      (accumulated as Qt = Q^T) is what one-sided Jacobi on the pair would
//      apply;
//   3. replaces Y by Qt Y over ncols_rot columns (streamed, 2 x 4 outputs per
//      thread, in place: a chunk is read whole before it is written).
// A pair whose fresh Gram matrix meets the stopping test (no rotation in the
// first inner sweep) is left as it is; a matrix is converged when a whole
// sweep rotates none of its pairs, the test of the row kernel on freshly
// formed inner products.  Padding rows (beyond `rows`) are zero, never
// rotated and never written.
constexpr int JP_B = 32;
constexpr int JP_R = 2 * JP_B;
constexpr int JP_KC = 32;             // columns per streamed chunk
constexpr int JP_LDT = JP_R + 4;      // Gram chunk, [column][row] (16-byte aligned rows)
constexpr int JP_LDA = JP_KC + 4;     // apply chunk, [row][column]
static_assert(JP_R == JPI_N, "the inner eigensolve is written for 64 x 64 Gram matrices");
static_assert((size_t)JP_KC * JP_LDT <= (size_t)JP_R * JPI_LDG && (size_t)JP_R * JP_LDA <= (size_t)JP_R * JPI_LDG,
              "the streamed chunks share the second Gram buffer");

// G0, G1 (the inner eigensolve's two Gram buffers; the streamed chunks of the
// Gram matrix and of the rotation reuse G1) and Qt
template <typename T>
size_t jacobi_pair_smem() {
    return (2 * (size_t)JP_R * JPI_LDG + (size_t)JP_R * JPI_LDQ) * sizeof(T) + 64;
}
template size_t jacobi_pair_smem<float>();
template size_t jacobi_pair_smem<double>();

__device__ __forceinline__ void jp_load4(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void jp_load4(const double* p, double* v) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256) jacobi_pair_kernel(const JacobiDescT<T>* __restrict__ descs,
                                                          const int4* __restrict__ tasks, int round, T tol,
                                                          int inner_max, int* __restrict__ rotated,
                                                          unsigned long long* __restrict__ rots,
                                                          unsigned long long* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char jp_raw[];
    T* G = reinterpret_cast<T*>(jp_raw);
    T* G1 = G + JP_R * JPI_LDG;
    T* Qt = G1 + JP_R * JPI_LDG;
    T* Yc = G1;  // streamed chunks (the inner eigensolve's second buffer is free then)
    __shared__ JpRound<T> jr[2];
    const int4 tk = tasks[blockIdx.x];
    const int mat = tk.x, kp = tk.y, nblk = tk.z;
    if (round >= nblk - 1) return;  // uniform over the CTA
    const JacobiDescT<T> d = descs[mat];
    int bp, bq;
    if (kp == 0) {
        bp = nblk - 1;
        bq = round;
    } else {
        bp = (round + kp) % (nblk - 1);
        bq = (round - kp + nblk - 1) % (nblk - 1);
    }
    const int tid = threadIdx.x;
    // global row of local row lr, -1 for padding
    auto grow = [&](int lr) -> int {
        const int r = (lr < JP_B ? bp : bq) * JP_B + (lr & (JP_B - 1));
        return r < d.rows ? r : -1;
    };
    const T absf = d.absfloor ? *d.absfloor : T(0);
    // stats: [0] pair tasks, [1] pairs rotated, [2..4] SM clock cycles of the
    // Gram matrix, the small eigensolve and the rotation of the rows (thread 0),
    // [5] inner sweeps
    const long long t0 = clock64();

    // ---- 1. Gram matrix over ncols_dot columns
    {
        const int ty = tid >> 4, tx = tid & 15;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        // software pipeline: the next chunk's values are loaded into registers
        // while the current chunk is multiplied out of shared memory
        constexpr int PER = JP_R * JP_KC / 256;  // values per thread and chunk
        const int kk_t = tid % JP_KC;
        int rows_t[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) rows_t[q] = grow((tid + 256 * q) / JP_KC);
        T pre[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q)
            pre[q] = (rows_t[q] >= 0 && kk_t < d.ncols_dot) ? __ldcg(d.A + (size_t)rows_t[q] * d.ld + kk_t) : T(0);
        for (int c0 = 0; c0 < d.ncols_dot; c0 += JP_KC) {
#pragma unroll
            for (int q = 0; q < PER; ++q) Yc[kk_t * JP_LDT + (tid + 256 * q) / JP_KC] = pre[q];
            __syncthreads();
            const int cn = c0 + JP_KC + kk_t;
#pragma unroll
            for (int q = 0; q < PER; ++q)
                pre[q] = (rows_t[q] >= 0 && cn < d.ncols_dot) ? __ldcg(d.A + (size_t)rows_t[q] * d.ld + cn) : T(0);
#pragma unroll 4
            for (int kk = 0; kk < JP_KC; ++kk) {
                T a[4], b[4];
                jp_load4(Yc + kk * JP_LDT + 4 * ty, a);
                jp_load4(Yc + kk * JP_LDT + 4 * tx, b);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) G[(4 * ty + i) * JPI_LDG + 4 * tx + j] = acc[i][j];
        for (int e = tid; e < JP_R * JP_R; e += 256) Qt[(e / JP_R) * JPI_LDQ + e % JP_R] = (e / JP_R == e % JP_R) ? T(1) : T(0);
        __syncthreads();
    }

    // ---- 2. two-sided cyclic Jacobi on G, rotations accumulated in Qt.  The
    // stopping test of the sweep (tol) on the fresh Gram matrix decides
    // whether the pair is rotated at all; once it is, up to inner_max inner
    // sweeps rotate couplings above a tighter inner test (tin, still well
    // above the rounding of G).  Whatever a visit leaves is met again by the
    // outer sweeps' test on fresh Gram matrices.
    const T ueps = sizeof(T) == 4 ? T(1.1920928955078125e-7) : T(2.220446049250313e-16);
    const T tin = fmax(tol * T(1.0 / 64.0), T(16) * ueps);
    const long long t1 = clock64();
    if (tid == 0) {
        atomicAdd(stats + 0, 1ull);
        atomicAdd(stats + 2, (unsigned long long)(t1 - t0));
    }
    {
        int mine = 0;
        for (int e = tid; e < JP_R * JP_R; e += 256) {
            const int p = e / JP_R, q = e % JP_R;
            if (q <= p) continue;
            const T a = G[p * JPI_LDG + p], b = G[q * JPI_LDG + q], g = G[p * JPI_LDG + q];
            if (g != T(0) && g * g > tol * tol * a * b && fabs(g) > absf) mine = 1;
        }
        if (!__syncthreads_or(mine)) return;  // the pair met the stopping test: rows unchanged
    }
    unsigned nrot = 0;
    const int inner = jpi_solve<T>(G, G1, Qt, jr, tin, absf, inner_max, nrot);
    if (nrot) atomicAdd(rots + mat, (unsigned long long)nrot);
    const long long t2 = clock64();
    if (tid == 0) {
        rotated[mat] = 1;
        atomicAdd(stats + 1, 1ull);
        atomicAdd(stats + 3, (unsigned long long)(t2 - t1));
        atomicAdd(stats + 5, (unsigned long long)inner);
    }

    // ---- 3. Y <- Qt Y over ncols_rot columns
    {
        const int ty = tid >> 3, tx = tid & 7;  // rows 2 ty, 2 ty + 1; columns 4 tx .. 4 tx + 3
        const int r0 = grow(2 * ty), r1 = grow(2 * ty + 1);
        constexpr int PER = JP_R * JP_KC / 256;
        const int kk_t = tid % JP_KC;
        int rows_t[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) rows_t[q] = grow((tid + 256 * q) / JP_KC);
        T pre[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q)
            pre[q] = (rows_t[q] >= 0 && kk_t < d.ncols_rot) ? __ldcg(d.A + (size_t)rows_t[q] * d.ld + kk_t) : T(0);
        for (int c0 = 0; c0 < d.ncols_rot; c0 += JP_KC) {
#pragma unroll
            for (int q = 0; q < PER; ++q) Yc[((tid + 256 * q) / JP_KC) * JP_LDA + kk_t] = pre[q];
            __syncthreads();
            // the next chunk is read before this one is written back: different
            // columns, so the in-place update stays safe
            const int cn = c0 + JP_KC + kk_t;
#pragma unroll
            for (int q = 0; q < PER; ++q)
                pre[q] = (rows_t[q] >= 0 && cn < d.ncols_rot) ? __ldcg(d.A + (size_t)rows_t[q] * d.ld + cn) : T(0);
            T o0[4] = {T(0), T(0), T(0), T(0)}, o1[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
            for (int k = 0; k < JP_R; ++k) {
                const T q0 = Qt[(2 * ty) * JPI_LDQ + k], q1 = Qt[(2 * ty + 1) * JPI_LDQ + k];
                T y[4];
                jp_load4(Yc + k * JP_LDA + 4 * tx, y);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    o0[j] = fma(q0, y[j], o0[j]);
                    o1[j] = fma(q1, y[j], o1[j]);
                }
            }
            __syncthreads();  // the chunk is read whole before the next one is loaded
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + 4 * tx + j;
                if (c < d.ncols_rot) {
                    if (r0 >= 0) d.A[(size_t)r0 * d.ld + c] = o0[j];
                    if (r1 >= 0) d.A[(size_t)r1 * d.ld + c] = o1[j];
                }
            }
        }
    }
    if (tid == 0) atomicAdd(stats + 4, (unsigned long long)(clock64() - t2));
}

template <typename T>
void launch_jacobi_pair_round(const JacobiDescT<T>* d, const int4* tasks, int ntasks, int round, T tol, int inner,
                              int* rotated, unsigned long long* rots, unsigned long long* stats, cudaStream_t s) {
    if (ntasks <= 0) return;
    const size_t smem = jacobi_pair_smem<T>();
    cudaFuncSetAttribute(jacobi_pair_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    jacobi_pair_kernel<T><<<ntasks, 256, smem, s>>>(d, tasks, round, tol, inner, rotated, rots, stats);
}
template void launch_jacobi_pair_round<float>(const JacobiDescT<float>*, const int4*, int, int, float, int, int*,
                                              unsigned long long*, unsigned long long*, cudaStream_t);
template void launch_jacobi_pair_round<double>(const JacobiDescT<double>*, const int4*, int, int, double, int, int*,
                                               unsigned long long*, unsigned long long*, cudaStream_t);

__global__ void or_flag_kernel(int* p, int bits) { atomicOr(p, bits); }
void launch_or_flag(int* p, int bits, cudaStream_t s) { or_flag_kernel<<<1, 1, 0, s>>>(p, bits); }

// ------------------------------------------------------------------ block Jacobi
// The same one-sided Jacobi with the rows resident in shared memory: the
// matrix is cut into 2 * JAC_CLUSTER row blocks of hb rows; in each block
// round every CTA of the cluster loads two blocks (P, Q) from global memory,
// performs all row pairs between them (hb sub-rounds of hb disjoint pairs,
// one warp per pair, __syncthreads between sub-rounds), and in the first
// block round also the pairs inside each block; it then writes the blocks
// back.  The blocks meet in a round-robin (circle) schedule, so one sweep
// visits every row pair once, with one cluster barrier per block round
// (2 * JAC_CLUSTER - 1 per sweep).  Row norms^2 are recomputed when a block is
// loaded and updated exactly after each rotation.
template <typename T, int CL>
__global__ void __launch_bounds__(1024)
    jacobi_block_kernel(const JacobiDescT<T>* __restrict__ descs, int max_sweeps, T tol, int* __restrict__ sweeps,
                        unsigned long long* __restrict__ rots, int* __restrict__ err, int report_noconv) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int mat = blockIdx.x / CL;
    const int crank = (int)cluster.block_rank();
    const JacobiDescT<T> d = descs[mat];
    constexpr int NBLK = 2 * CL;
    const int hb = (d.rows + NBLK - 1) / NBLK;
    const int W = d.ncols_rot, D = d.ncols_dot;
    T* blk = reinterpret_cast<T*>(jac_smem);  // [2][hb][W]
    T* nrm = blk + (size_t)2 * hb * W;        // [2][hb]
    __shared__ int rotated;
    __shared__ T jg[JAC_MAX_PAIRS], jcs[JAC_MAX_PAIRS], jsn[JAC_MAX_PAIRS];
    __shared__ int jflag[JAC_MAX_PAIRS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int hbe = hb + (hb & 1);
    const T absf = d.absfloor ? *d.absfloor : T(0);
    unsigned long long my_rots = 0;
    int sweep = 0;
    bool done = false;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        for (int br = 0; br < NBLK - 1; ++br) {
            int P, Q;
            if (crank == 0) {
                P = NBLK - 1;
                Q = br;
            } else {
                P = (br + crank) % (NBLK - 1);
                Q = (br - crank + NBLK - 1) % (NBLK - 1);
            }
            const int r0[2] = {P * hb, Q * hb};
            int nr[2];
            for (int k = 0; k < 2; ++k) nr[k] = max(0, min(hb, d.rows - r0[k]));
            for (int k = 0; k < 2; ++k)
                for (int r = warp; r < nr[k]; r += nwarps) {
                    const T* src = d.A + (size_t)(r0[k] + r) * d.ld;
                    T* dst = blk + ((size_t)k * hb + r) * W;
                    T a = T(0);
                    for (int c = lane; c < W; c += 32) {
                        const T v = __ldcg(src + c);
                        dst[c] = v;
                        if (c < D) a = fma(v, v, a);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    if (lane == 0) nrm[k * hb + r] = a;
                }
            __syncthreads();
            // One sub-round in three phases: inner products (one warp per pair),
            // rotation parameters and norm updates (one thread per pair), then
            // the rotations (one warp per pair).  The scalar rotation math runs
            // once per pair instead of on every lane.
            auto subround = [&](int npairs, auto&& pair_of) {
                for (int k = warp; k < npairs; k += nwarps) {
                    int sa, sb;
                    if (!pair_of(k, sa, sb)) continue;
                    const T* xp = blk + (size_t)sa * W;
                    const T* xq = blk + (size_t)sb * W;
                    T g0 = T(0), g1 = T(0);
                    int c = lane;
                    for (; c + 32 < D; c += 64) {
                        g0 = fma(xp[c], xq[c], g0);
                        g1 = fma(xp[c + 32], xq[c + 32], g1);
                    }
                    if (c < D) g0 = fma(xp[c], xq[c], g0);
                    T g = g0 + g1;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                    if (lane == 0) jg[k] = g;
                }
                __syncthreads();
                if ((int)threadIdx.x < npairs) {
                    const int k = threadIdx.x;
                    int sa, sb;
                    jflag[k] = 0;
                    if (pair_of(k, sa, sb)) {
                        const T g = jg[k], a = nrm[sa], b = nrm[sb];
                        if (g != T(0) && g * g > tol * tol * a * b && fabs(g) > absf) {
                            T cs, sn, t;
                            jac_rotation(a, b, g, cs, sn, t);
                            jcs[k] = cs;
                            jsn[k] = sn;
                            jflag[k] = 1;
                            nrm[sa] = fma(-t, g, a);
                            nrm[sb] = fma(t, g, b);
                            ++my_rots;
                            rotated = 1;
                        }
                    }
                }
                __syncthreads();
                for (int k = warp; k < npairs; k += nwarps) {
                    if (!jflag[k]) continue;
                    int sa, sb;
                    pair_of(k, sa, sb);
                    T* xp = blk + (size_t)sa * W;
                    T* xq = blk + (size_t)sb * W;
                    const T cs = jcs[k], sn = jsn[k];
                    for (int c = lane; c < W; c += 32) {
                        const T u = xp[c], v = xq[c];
                        xp[c] = fma(cs, u, -sn * v);
                        xq[c] = fma(sn, u, cs * v);
                    }
                }
                __syncthreads();
            };
            if (br == 0) {
                // pairs inside each of the two blocks (circle schedule on hbe)
                for (int sr = 0; sr < hbe - 1; ++sr)
                    subround(hbe, [&](int k, int& sa, int& sb) {
                        const int which = k / (hbe / 2), kk = k % (hbe / 2);
                        int a, b;
                        if (kk == 0) {
                            a = hbe - 1;
                            b = sr;
                        } else {
                            a = (sr + kk) % (hbe - 1);
                            b = (sr - kk + (hbe - 1)) % (hbe - 1);
                        }
                        sa = which * hb + a;
                        sb = which * hb + b;
                        return a < nr[which] && b < nr[which];
                    });
            }
            // pairs between the two blocks
            for (int sr = 0; sr < hb; ++sr)
                subround(hb, [&](int a, int& sa, int& sb) {
                    const int b = (a + sr) % hb;
                    sa = a;
                    sb = hb + b;
                    return a < nr[0] && b < nr[1];
                });
            for (int k = 0; k < 2; ++k)
                for (int r = warp; r < nr[k]; r += nwarps) {
                    T* dst = d.A + (size_t)(r0[k] + r) * d.ld;
                    const T* src = blk + ((size_t)k * hb + r) * W;
                    for (int c = lane; c < W; c += 32) dst[c] = src[c];
                }
            __threadfence();
            cluster.sync();
        }
        int any = 0;
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) any |= *cluster.map_shared_rank(&rotated, rr);
        cluster.sync();
        if (!any) {
            done = true;
            break;
        }
    }
    if (my_rots) atomicAdd(rots + mat, my_rots);
    if (crank == 0 && threadIdx.x == 0) {
        sweeps[mat] = done ? sweep + 1 : sweep;
        if (!done && report_noconv) atomicOr(err, DERR_EIG_NOCONV);
    }
}

template <typename T>
size_t jacobi_block_smem(int rows, int ncols_rot, int cluster) {
    const size_t hb = (size_t)(rows + 2 * cluster - 1) / (2 * cluster);
    return (2 * hb * (size_t)ncols_rot + 2 * hb) * sizeof(T);
}
template size_t jacobi_block_smem<float>(int, int, int);
template size_t jacobi_block_smem<double>(int, int, int);

// One launch of the block kernel with a cluster of CL CTAs per matrix
// (cluster dimension given at launch; CL = 16 is the non-portable size).
// Returns false, with nothing launched, when the blocks do not fit or the
// device cannot co-schedule such a cluster.
template <typename T, int CL>
bool launch_jacobi_block_cl(const JacobiDescT<T>* d, int nmat, size_t smem, int max_rows, int max_sweeps, T tol,
                            int* sweeps, unsigned long long* rots, int* err, int report_noconv, cudaStream_t s) {
    if (smem > JAC_BLOCK_SMEM_MAX) return false;
    const int hb = (max_rows + 2 * CL - 1) / (2 * CL);
    if (hb + 2 > JAC_MAX_PAIRS) return false;
    auto kern = jacobi_block_kernel<T, CL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (CL > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    // one warp per pair of a sub-round (hb pairs), 8 to 32 warps
    const int warps = hb < 8 ? 8 : (hb > 32 ? 32 : hb);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nmat * CL);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return false;
    }
    if (cudaLaunchKernelEx(&cfg, kern, d, max_sweeps, tol, sweeps, rots, err, report_noconv) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T>
bool launch_jacobi_block(const JacobiDescT<T>* d, int nmat, size_t smem8, size_t smem16, int max_rows,
                         int max_sweeps, T tol, int* sweeps, unsigned long long* rots, int* err, int report_noconv,
                         cudaStream_t s) {
    if (nmat <= 0) return true;
    if (launch_jacobi_block_cl<T, JAC_CLUSTER>(d, nmat, smem8, max_rows, max_sweeps, tol, sweeps, rots, err,
                                               report_noconv, s))
        return true;
    return launch_jacobi_block_cl<T, 2 * JAC_CLUSTER>(d, nmat, smem16, max_rows, max_sweeps, tol, sweeps, rots, err,
                                                      report_noconv, s);
}
template bool launch_jacobi_block<float>(const JacobiDescT<float>*, int, size_t, size_t, int, int, float, int*,
                                         unsigned long long*, int*, int, cudaStream_t);
template bool launch_jacobi_block<double>(const JacobiDescT<double>*, int, size_t, size_t, int, int, double, int*,
                                          unsigned long long*, int*, int, cudaStream_t);

// absfloor[mat] = eps * max_r ||row r||^2 over ncols_dot (one CTA per matrix).
template <typename T>
__global__ void __launch_bounds__(256) row_maxnorm2_kernel(const JacobiDescT<T>* __restrict__ descs, T eps,
                                                            T* __restrict__ out) {
    const JacobiDescT<T> d = descs[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ T wmax[8];
    T mx = T(0);
    for (int r = warp; r < d.rows; r += 8) {
        const T* x = d.A + (size_t)r * d.ld;
        T a = T(0);
        for (int c = lane; c < d.ncols_dot; c += 32) a = fma(x[c], x[c], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        mx = a > mx ? a : mx;
    }
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = T(0);
        for (int w = 0; w < 8; ++w) m = wmax[w] > m ? wmax[w] : m;
        out[blockIdx.x] = eps * m;
    }
}

template <typename T>
void launch_row_maxnorm2(const JacobiDescT<T>* d, int nmat, T eps, T* out, cudaStream_t s) {
    if (nmat > 0) row_maxnorm2_kernel<T><<<nmat, 256, 0, s>>>(d, eps, out);
}
template void launch_row_maxnorm2<float>(const JacobiDescT<float>*, int, float, float*, cudaStream_t);
template void launch_row_maxnorm2<double>(const JacobiDescT<double>*, int, double, double*, cudaStream_t);

// out32 (rows x (L + rows), ld L + rows) = [float(A) | I] for A rows x L (lda).
__global__ void to_f32_with_identity_kernel(const CvtDesc* __restrict__ descs) {
    const CvtDesc d = descs[blockIdx.y];
    const int w = d.L + d.rows;
    for (int r = blockIdx.x; r < d.rows; r += gridDim.x) {
        const double* a = d.A + (size_t)r * d.lda;
        float* o = d.out32 + (size_t)r * w;
        for (int c = threadIdx.x; c < w; c += blockDim.x) o[c] = (c < d.L) ? (float)a[c] : (c - d.L == r ? 1.f : 0.f);
    }
}

void launch_to_f32_with_identity(const CvtDesc* d, int nmat, int maxrows, cudaStream_t s) {
    if (nmat <= 0 || maxrows <= 0) return;
    dim3 grid(min(maxrows, 1024), nmat);
    to_f32_with_identity_kernel<<<grid, 256, 0, s>>>(d);
}

// Q64 (rows x rows) = double(right block of out32).
__global__ void extract_q_kernel(const CvtDesc* __restrict__ descs) {
    const CvtDesc d = descs[blockIdx.y];
    const int w = d.L + d.rows;
    for (int r = blockIdx.x; r < d.rows; r += gridDim.x) {
        const float* o = d.out32 + (size_t)r * w + d.L;
        double* q = d.Q + (size_t)r * d.rows;
        for (int c = threadIdx.x; c < d.rows; c += blockDim.x) q[c] = (double)o[c];
    }
}

void launch_extract_q(const CvtDesc* d, int nmat, int maxrows, cudaStream_t s) {
    if (nmat <= 0 || maxrows <= 0) return;
    dim3 grid(min(maxrows, 1024), nmat);
    extract_q_kernel<<<grid, 256, 0, s>>>(d);
}

// Row norms over ncols_dot (written as double), delta = eps * max norm,
// optional row scaling by 1/sqrt(norm) over ncols_rot.  One CTA per matrix,
// one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) rownorms_kernel(const JacobiDescT<T>* __restrict__ descs,
                                                        double* const* __restrict__ sig, T* __restrict__ delta,
                                                        double eps, int scale_rows) {
    const JacobiDescT<T> d = descs[blockIdx.x];
    double* out = sig[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ T wmax[8];
    T mx = T(0);
    for (int r = warp; r < d.rows; r += 8) {
        T* row = d.A + (size_t)r * d.ld;
        T s = T(0);
        for (int c = lane; c < d.ncols_dot; c += 32) s = fma(row[c], row[c], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const T nrm = sqrt(s);
        if (lane == 0) out[r] = (double)nrm;
        mx = fmax(mx, nrm);
        if (scale_rows && nrm > T(0)) {
            const T f = rsqrt_t(nrm);
            for (int c = lane; c < d.ncols_rot; c += 32) row[c] *= f;
        }
    }
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = T(0);
        for (int w = 0; w < 8; ++w) m = fmax(m, wmax[w]);
        if (delta) delta[blockIdx.x] = (T)(eps * (double)m);
    }
}

template <typename T>
void launch_rownorms(const JacobiDescT<T>* d, int nmat, double* const* sigma_ptrs, T* delta, double eps,
                     int scale_rows, cudaStream_t s) {
    if (nmat > 0) rownorms_kernel<T><<<nmat, 256, 0, s>>>(d, sigma_ptrs, delta, eps, scale_rows);
}
template void launch_rownorms<float>(const JacobiDescT<float>*, int, double* const*, float*, double, int,
                                     cudaStream_t);
template void launch_rownorms<double>(const JacobiDescT<double>*, int, double* const*, double*, double, int,
                                      cudaStream_t);

__global__ void __launch_bounds__(256) diag_basis_kernel(const DiagBasisDesc* __restrict__ descs) {
    const DiagBasisDesc d = descs[blockIdx.y];
    const int k = blockIdx.x;
    if (k >= d.nI) return;
    double* row = d.Zt + (size_t)k * d.nI;
    for (int c = threadIdx.x; c < d.nI; c += blockDim.x)
        row[c] = (c == k) ? 1.0 / sqrt(d.A[(size_t)k * d.lda + k]) : 0.0;
}

void launch_diag_basis(const DiagBasisDesc* d, int nmat, int maxn, cudaStream_t s) {
    if (nmat > 0 && maxn > 0) diag_basis_kernel<<<dim3(maxn, nmat), 256, 0, s>>>(d);
}

__global__ void __launch_bounds__(256) diag_scale_kernel(const DiagScaleDesc* __restrict__ descs) {
    const DiagScaleDesc d = descs[blockIdx.y];
    const int r = blockIdx.x;
    if (r >= d.ni) return;
    const double* a = d.A + (size_t)r * d.ni;
    const double fr = r < d.nI ? 1.0 / sqrt(d.A[(size_t)r * d.ni + r]) : 0.0;
    for (int c = threadIdx.x; c < d.nI; c += blockDim.x) {
        const double az = a[c] * (1.0 / sqrt(d.A[(size_t)c * d.ni + c]));
        d.AZ[(size_t)r * d.nI + c] = az;
        if (r < d.nI && c <= r) d.Eii[(size_t)r * d.ldE + c] = fr * az;
    }
}

void launch_diag_scale(const DiagScaleDesc* d, int nmat, int maxni, cudaStream_t s) {
    if (nmat > 0 && maxni > 0) diag_scale_kernel<<<dim3(maxni, nmat), 256, 0, s>>>(d);
}

__global__ void __launch_bounds__(256) mf_prepare_kernel(const MfPrepDesc* __restrict__ descs) {
    const MfPrepDesc d = descs[blockIdx.y];
    const int r = blockIdx.x;
    if (r >= d.ni) return;
    const double f = 1.0 / (d.sig[r] + *d.delta);
    const double* x = d.X1 + (size_t)r * d.ld + d.nR;
    for (int c = threadIdx.x; c < d.nI; c += blockDim.x) {
        const double v = x[c];
        d.Cc[(size_t)r * d.nI + c] = v;
        d.Bm[(size_t)r * d.nI + c] = v * f;
    }
}

void launch_mf_prepare(const MfPrepDesc* d, int nmat, int maxni, cudaStream_t s) {
    if (nmat > 0 && maxni > 0) mf_prepare_kernel<<<dim3(maxni, nmat), 256, 0, s>>>(d);
}

template <typename T>
__global__ void __launch_bounds__(256) build_kjac_kernel(const KjacDesc<T>* __restrict__ descs) {
    const KjacDesc<T> d = descs[blockIdx.y];
    const int r = blockIdx.x;
    if (r >= d.ni) return;
    const T* c = d.C + (size_t)r * d.ldc;
    T* j = d.J + (size_t)r * d.ldj;
    for (int k = threadIdx.x; k < d.nR + d.ni; k += blockDim.x)
        j[k] = k < d.nR ? c[k] : (k - d.nR == r ? T(1) : T(0));
}

template <typename T>
void launch_build_kjac(const KjacDesc<T>* d, int nmat, int maxrows, cudaStream_t s) {
    if (nmat > 0 && maxrows > 0) build_kjac_kernel<T><<<dim3(maxrows, nmat), 256, 0, s>>>(d);
}
template void launch_build_kjac<float>(const KjacDesc<float>*, int, int, cudaStream_t);
template void launch_build_kjac<double>(const KjacDesc<double>*, int, int, cudaStream_t);

// one warp per row: s^2 over the first nR entries, then the right part
// scaled by 1 / sqrt(s^2 + delta)
template <typename T>
__global__ void __launch_bounds__(256) kjac_scale_kernel(const KjacDesc<T>* __restrict__ descs) {
    const KjacDesc<T> d = descs[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T dl = *d.delta;
    for (int r = warp; r < d.ni; r += 8) {
        T* row = d.J + (size_t)r * d.ldj;
        T s2 = T(0);
        for (int k = lane; k < d.nR; k += 32) s2 = fma(row[k], row[k], s2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const T f = T(1) / sqrt(s2 + dl);
        for (int k = d.nR + lane; k < d.nR + d.ni; k += 32) row[k] *= f;
    }
}

template <typename T>
void launch_kjac_scale(const KjacDesc<T>* d, int nmat, cudaStream_t s) {
    if (nmat > 0) kjac_scale_kernel<T><<<nmat, 256, 0, s>>>(d);
}
template void launch_kjac_scale<float>(const KjacDesc<float>*, int, cudaStream_t);
template void launch_kjac_scale<double>(const KjacDesc<double>*, int, cudaStream_t);

template <typename T>
__global__ void add_diag_kernel(T* const* __restrict__ mats, const int* __restrict__ n, const int* __restrict__ ld,
                                const T* __restrict__ delta) {
    const int b = blockIdx.y;
    T* M = mats[b];
    const T dv = delta[b];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n[b]; j += gridDim.x * blockDim.x)
        M[(size_t)j * ld[b] + j] += dv;
}

template <typename T>
void launch_add_diag(T* const* mats, const int* n, const int* ld, const T* delta, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid((maxn + 255) / 256, nmat);
    add_diag_kernel<T><<<grid, 256, 0, s>>>(mats, n, ld, delta);
}
template void launch_add_diag<float>(float* const*, const int*, const int*, const float*, int, int, cudaStream_t);
template void launch_add_diag<double>(double* const*, const int*, const int*, const double*, int, int,
                                      cudaStream_t);

template <typename T>
__global__ void mirror_lower_kernel(T* const* __restrict__ mats, const int* __restrict__ n,
                                    const int* __restrict__ ld) {
    const int b = blockIdx.y;
    T* M = mats[b];
    const int nn = n[b], l = ld[b];
    for (int r = blockIdx.x; r < nn; r += gridDim.x)
        for (int c = r + 1 + threadIdx.x; c < nn; c += blockDim.x) M[(size_t)r * l + c] = M[(size_t)c * l + r];
}

template <typename T>
void launch_mirror_lower(T* const* mats, const int* n, const int* ld, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid(min(maxn, 1024), nmat);
    mirror_lower_kernel<T><<<grid, 128, 0, s>>>(mats, n, ld);
}
template void launch_mirror_lower<float>(float* const*, const int*, const int*, int, int, cudaStream_t);
template void launch_mirror_lower<double>(double* const*, const int*, const int*, int, int, cudaStream_t);

// dst = src^T for square n x n matrices, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void transpose_kernel(const T* const* __restrict__ src, T* const* __restrict__ dst,
                                 const int* __restrict__ n, const int* __restrict__ lds,
                                 const int* __restrict__ ldd) {
    const int b = blockIdx.z;
    const int nn = n[b];
    const int nt = (nn + 31) / 32;
    __shared__ T tile[32][33];
    for (int t = blockIdx.x; t < nt * nt; t += gridDim.x) {
        const int tr = t / nt, tc = t % nt;
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int r = e / 32, c = e % 32;
            const int gr = tr * 32 + r, gc = tc * 32 + c;
            tile[r][c] = (gr < nn && gc < nn) ? src[b][(size_t)gr * lds[b] + gc] : T(0);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int r = e / 32, c = e % 32;
            const int gr = tc * 32 + r, gc = tr * 32 + c;
            if (gr < nn && gc < nn) dst[b][(size_t)gr * ldd[b] + gc] = tile[c][r];
        }
        __syncthreads();
    }
}

template <typename T>
void launch_transpose(const T* const* src, T* const* dst, const int* n, const int* lds, const int* ldd, int nmat,
                      int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    const int nt = (maxn + 31) / 32;
    dim3 grid(min(nt * nt, 4096), 1, nmat);
    transpose_kernel<T><<<grid, 256, 0, s>>>(src, dst, n, lds, ldd);
}
template void launch_transpose<float>(const float* const*, float* const*, const int*, const int*, const int*, int,
                                      int, cudaStream_t);
template void launch_transpose<double>(const double* const*, double* const*, const int*, const int*, const int*,
                                       int, int, cudaStream_t);

// dst = src^T for a batch of rectangular FP64 matrices, 32 x 32 tiles through
// shared memory (blockIdx.z = matrix)
__global__ void transpose_rect_kernel(const TransDesc* __restrict__ descs) {
    const TransDesc d = descs[blockIdx.z];
    __shared__ double tile[32][33];
    const int tr = (d.rows + 31) / 32, tc = (d.cols + 31) / 32;
    for (int t = blockIdx.x; t < tr * tc; t += gridDim.x) {
        const int r0 = (t / tc) * 32, c0 = (t % tc) * 32;
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int r = e / 32, c = e % 32;
            tile[r][c] = (r0 + r < d.rows && c0 + c < d.cols) ? d.src[(size_t)(r0 + r) * d.lds + c0 + c] : 0.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int c = e / 32, r = e % 32;
            if (r0 + r < d.rows && c0 + c < d.cols) d.dst[(size_t)(c0 + c) * d.ldd + r0 + r] = tile[r][c];
        }
        __syncthreads();
    }
}

void launch_transpose_rect(const TransDesc* d, int nmat, int maxdim, cudaStream_t s) {
    if (nmat <= 0 || maxdim <= 0) return;
    const int t = (maxdim + 31) / 32;
    dim3 grid(min(t * t, 4096), 1, nmat);
    transpose_rect_kernel<<<grid, 256, 0, s>>>(d);
}

// dst[i] = (To) src[i]
template <typename Ti, typename To>
__global__ void convert_kernel(const Ti* __restrict__ src, To* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (To)src[i];
}

template <typename Ti, typename To>
void launch_convert(const Ti* src, To* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t want = (n + 255) / 256;
    convert_kernel<Ti, To><<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(src, dst, n);
}
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);

// dst_b[r * ldd_b + c] = (To) src_b[r * lds_b + c] for r, c < n_b (batch b = blockIdx.y)
template <typename Ti, typename To>
__global__ void convert_blocks_kernel(const Ti* const* __restrict__ src, const int* __restrict__ lds,
                                      To* const* __restrict__ dst, const int* __restrict__ ldd,
                                      const int* __restrict__ n) {
    const int b = blockIdx.y;
    const int nn = n[b];
    const Ti* S = src[b];
    To* D = dst[b];
    for (int r = blockIdx.x; r < nn; r += gridDim.x)
        for (int c = threadIdx.x; c < nn; c += blockDim.x) D[(size_t)r * ldd[b] + c] = (To)S[(size_t)r * lds[b] + c];
}

template <typename Ti, typename To>
void launch_convert_blocks(const Ti* const* src, const int* lds, To* const* dst, const int* ldd, const int* n,
                           int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid(min(maxn, 1024), nmat);
    convert_blocks_kernel<Ti, To><<<grid, 256, 0, s>>>(src, lds, dst, ldd, n);
}
template void launch_convert_blocks<double, float>(const double* const*, const int*, float* const*, const int*,
                                                   const int*, int, int, cudaStream_t);

// ------------------------------------------------------------------ tridiagonal eigenvalues
// Householder reduction of a symmetric n x n matrix (full storage, updated in
// place) to tridiagonal form T = Q^T A Q, one CTA per matrix: at step k the
// reflector H = I - beta v v^T maps A[k+1:, k] onto alpha e_1, and the trailing
// block becomes H A22 H = A22 - v w^T - w v^T with p = beta A22 v,
// w = p - (beta/2)(p^T v) v.  Output: diagonal d[0..n) and sub-diagonal
// e[1..n) (e[0] = 0).
// A cluster of JAC_CLUSTER CTAs reduces one matrix; row r of the matrix
// belongs to CTA r mod JAC_CLUSTER.  Per step: partial sums of the column norm
// (cluster barrier 1, partials read through distributed shared memory), the
// owned entries of p = beta A22 v written to a global buffer with partial sums
// of p^T v (barrier 2), the full w = p - K v rebuilt in shared memory and the
// owned rows updated (barrier 3).  All CTAs compute the same reflector from the
// same partials in the same order, so every barrier is reached by every
// thread.
template <typename T>
__global__ void __cluster_dims__(JAC_CLUSTER, 1, 1) __launch_bounds__(256)
    tridiag_kernel(const TridiagDescT<T>* __restrict__ descs) {
    cg::cluster_group cluster = cg::this_cluster();
    const int mat = blockIdx.x / JAC_CLUSTER;
    const int crank = (int)cluster.block_rank();
    const TridiagDescT<T> t = descs[mat];
    const int n = t.n;
    extern __shared__ __align__(16) unsigned char tri_smem_raw[];
    T* v = reinterpret_cast<T*>(tri_smem_raw);  // n
    T* w = v + n;     // n
    __shared__ T part[2];
    __shared__ T red[8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    T* A = t.A;
    if (crank == 0 && tid == 0) t.e[0] = T(0);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        // owned rows of the trailing block: global rows r = k+1+i with r % CS == crank
        const int first = (k + 1) + ((crank - (k + 1)) % JAC_CLUSTER + JAC_CLUSTER) % JAC_CLUSTER;
        T sl = T(0);
        for (int r = first + JAC_CLUSTER * tid; r < n; r += JAC_CLUSTER * blockDim.x) {
            const T x = __ldcg(A + (size_t)r * t.ld + k);
            sl = fma(x, x, sl);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
        if (lane == 0) red[warp] = sl;
        __syncthreads();
        if (tid == 0) {
            T q = T(0);
            for (int ww = 0; ww < nw; ++ww) q += red[ww];
            part[0] = q;
        }
        cluster.sync();  // 1
        T s2 = T(0);
        for (int rr = 0; rr < JAC_CLUSTER; ++rr) s2 += *cluster.map_shared_rank(&part[0], rr);
        const T x0 = __ldcg(A + (size_t)(k + 1) * t.ld + k);
        const T tail = s2 - x0 * x0;
        if (crank == 0 && tid == 0) t.d[k] = __ldcg(A + (size_t)k * t.ld + k);
        if (!(tail > T(0))) {
            if (crank == 0 && tid == 0) t.e[k + 1] = x0;
            cluster.sync();  // 2
            cluster.sync();  // 3
            continue;
        }
        const T alpha = -copysign(sqrt(s2), x0);
        const T v0 = x0 - alpha;
        const T beta = T(2) / fma(v0, v0, tail);
        for (int i = tid; i < m; i += blockDim.x) v[i] = (i == 0) ? v0 : __ldcg(A + (size_t)(k + 1 + i) * t.ld + k);
        __syncthreads();
        // p = beta A22 v for owned rows
        T kl = T(0);
        for (int r = first + JAC_CLUSTER * warp; r < n; r += JAC_CLUSTER * nw) {
            const T* row = A + (size_t)r * t.ld + (k + 1);
            T acc0 = T(0), acc1 = T(0);
            int j = lane;
            for (; j + 32 < m; j += 64) {
                acc0 = fma(__ldcg(row + j), v[j], acc0);
                acc1 = fma(__ldcg(row + j + 32), v[j + 32], acc1);
            }
            if (j < m) acc0 = fma(__ldcg(row + j), v[j], acc0);
            T acc = acc0 + acc1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const int i = r - (k + 1);
            if (lane == 0) {
                t.p[i] = beta * acc;
                kl = fma(beta * acc, v[i], kl);
            }
        }
        if (lane == 0) red[warp] = kl;
        __syncthreads();
        if (tid == 0) {
            T q = T(0);
            for (int ww = 0; ww < nw; ++ww) q += red[ww];
            part[1] = q;
        }
        __threadfence();
        cluster.sync();  // 2
        T ks = T(0);
        for (int rr = 0; rr < JAC_CLUSTER; ++rr) ks += *cluster.map_shared_rank(&part[1], rr);
        const T K = T(0.5) * beta * ks;
        for (int i = tid; i < m; i += blockDim.x) w[i] = fma(-K, v[i], __ldcg(t.p + i));
        __syncthreads();
        for (int r = first + JAC_CLUSTER * warp; r < n; r += JAC_CLUSTER * nw) {
            T* row = A + (size_t)r * t.ld + (k + 1);
            const int i = r - (k + 1);
            const T vi = v[i], wi = w[i];
            for (int j = lane; j < m; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], __ldcg(row + j)));
        }
        if (crank == 0 && tid == 0) t.e[k + 1] = alpha;
        __threadfence();
        cluster.sync();  // 3
    }
    if (crank == 0 && tid == 0) {
        if (n >= 2) {
            t.d[n - 2] = __ldcg(A + (size_t)(n - 2) * t.ld + (n - 2));
            t.e[n - 1] = __ldcg(A + (size_t)(n - 1) * t.ld + (n - 2));
        }
        if (n >= 1) t.d[n - 1] = __ldcg(A + (size_t)(n - 1) * t.ld + (n - 1));
    }
}

// The same reduction with the matrix held in distributed shared memory: a
// cluster of TD_CL CTAs per matrix, CTA c keeping the lower-triangle part
// (columns 0..r) of the rows r = c mod TD_CL, packed row after row.  Per step
// k (m = n - k - 1 trailing rows):
//   A. the owned entries of column k go to colk and their squares to a partial
//      sum; the owner of row k writes d[k];                 (cluster barrier 1)
//   B. the norm, alpha and beta from the TD_CL partials in rank order; v
//      gathered from the owners' colk; for every owned row r (one warp) the
//      row part sum_{j <= r} A_rj v_j of (A22 v)_r and, for j < r, the column
//      part A_rj v_r, accumulated per warp (in row order) and then summed over
//      the warps into pcs;                                  (cluster barrier 2)
//   C. p_r = beta (row part + the TD_CL column parts of r in rank order) for
//      the owned rows, and a partial sum of p^T v;          (cluster barrier 3)
//   D. K = beta/2 p^T v, w = p - K v gathered from the owners, and the rank-2
//      update A_rj -= v_r w_j + w_r v_j of the owned rows.
// colk, pcs, pv and the partials are double-buffered by step parity, so the
// three barriers of a step also order it against the next one.  Every
// reduction has a fixed order: the result does not depend on the schedule.
constexpr int TD_CL = 16;

__host__ __device__ inline int64_t td_rows_entries(int c, int n, int* nown_out = nullptr) {
    const int nown = c < n ? (n - c + TD_CL - 1) / TD_CL : 0;
    if (nown_out) *nown_out = nown;
    return (int64_t)nown * (c + 1) + (int64_t)(TD_CL / 2) * nown * (nown - 1);
}

// Entries of the packed-row region, the same in every CTA of the cluster (the
// largest share, rounded up to even), so that the vectors after it, which
// other CTAs read, sit at the same offset in every CTA.
__host__ __device__ inline int64_t td_region(int n) {
    int64_t mx = 0;
    for (int c = 0; c < TD_CL; ++c) {
        const int64_t e = td_rows_entries(c, n);
        mx = e > mx ? e : mx;
    }
    return (mx + 1) / 2 * 2;
}
// the packed rows, then colk, pcs, pv (2n each), v, w (n each), pcw (8n)
constexpr int TD_VECS = 16;

template <typename T>
size_t tridiag_dsm_smem(int n) {
    return (size_t)(td_region(n) + TD_VECS * (int64_t)n) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(256) tridiag_dsm_kernel(const TridiagDescT<T>* __restrict__ descs) {
    cg::cluster_group cluster = cg::this_cluster();
    const int mat = blockIdx.x / TD_CL;
    const int c = (int)cluster.block_rank();
    const TridiagDescT<T> t = descs[mat];
    const int n = t.n;
    extern __shared__ __align__(16) unsigned char td_raw[];
    int nown = 0;
    (void)td_rows_entries(c, n, &nown);
    T* L = reinterpret_cast<T*>(td_raw);
    T* colk = L + td_region(n);  // 2n, by global row
    T* pcs = colk + 2 * n;            // 2n, by global row
    T* pv = pcs + 2 * n;              // 2n, by global row
    T* v = pv + 2 * n;                // n, by trailing index
    T* w = v + n;                     // n
    T* pcw = w + n;                   // 8n: column parts per warp
    __shared__ T part[2][2];
    __shared__ T red[8];
    __shared__ T scal[4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto off = [&](int l) -> int64_t { return (int64_t)l * (c + 1) + (int64_t)(TD_CL / 2) * l * (l - 1); };
    // sum of the TD_CL partials part[b][q] in rank order, by warp 0, into scal[slot]
    auto cluster_sum = [&](int b, int q, int slot) {
        if (warp == 0) {
            T x = T(0);
            if (lane < TD_CL) x = *cluster.map_shared_rank(&part[b][q], lane);
            T acc = T(0);
            for (int i = 0; i < TD_CL; ++i) acc += __shfl_sync(0xffffffffu, x, i);
            if (lane == 0) scal[slot] = acc;
        }
        __syncthreads();
    };
    auto block_sum = [&](T x, int b, int q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (tid == 0) {
            T acc = T(0);
            for (int ww = 0; ww < 8; ++ww) acc += red[ww];
            part[b][q] = acc;
        }
    };

    for (int l = 0; l < nown; ++l) {
        const int r = c + TD_CL * l;
        T* dst = L + off(l);
        for (int j = tid; j <= r; j += blockDim.x) dst[j] = t.A[(size_t)r * t.ld + j];
    }
    if (c == 0 && tid == 0) t.e[0] = T(0);
    __syncthreads();

    for (int k = 0; k + 2 < n; ++k) {
        const int b = k & 1, m = n - k - 1;
        const int l0 = (k + 1 - c) > 0 ? (k + 1 - c + TD_CL - 1) / TD_CL : 0;
        T* colb = colk + (size_t)b * n;
        T* pcb = pcs + (size_t)b * n;
        T* pvb = pv + (size_t)b * n;
        // A
        T sl = T(0);
        for (int l = l0 + tid; l < nown; l += blockDim.x) {
            const int r = c + TD_CL * l;
            const T x = L[off(l) + k];
            colb[r] = x;
            sl = fma(x, x, sl);
        }
        if (c == k % TD_CL && tid == 0) t.d[k] = L[off((k - c) / TD_CL) + k];
        block_sum(sl, b, 0);
        cluster.sync();  // 1
        // B
        cluster_sum(b, 0, 0);
        const T s2 = scal[0];
        const T x0 = *cluster.map_shared_rank(colb + (k + 1), (k + 1) % TD_CL);
        const T tail = s2 - x0 * x0;
        if (!(tail > T(0))) {
            if (c == 0 && tid == 0) t.e[k + 1] = x0;
            __syncthreads();
            continue;
        }
        const T alpha = -copysign(sqrt(s2), x0);
        const T v0 = x0 - alpha;
        const T beta = T(2) / fma(v0, v0, tail);
        for (int i = tid; i < m; i += blockDim.x) {
            const int r = k + 1 + i;
            v[i] = i == 0 ? v0 : *cluster.map_shared_rank(colb + r, r % TD_CL);
        }
        T* pw = pcw + (size_t)warp * n;
        for (int j = lane; j < m; j += 32) pw[j] = T(0);
        __syncthreads();
        for (int l = l0 + warp; l < nown; l += 8) {
            const int r = c + TD_CL * l, i = r - k - 1;
            const T* row = L + off(l) + (k + 1);
            const T vi = v[i];
            T acc = T(0);
            for (int j = lane; j <= i; j += 32) {
                const T a = row[j];
                acc = fma(a, v[j], acc);
                if (j < i) pw[j] = fma(a, vi, pw[j]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) pvb[r] = acc;
        }
        __syncthreads();
        for (int j = tid; j < m; j += blockDim.x) {
            T acc = T(0);
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) acc += pcw[(size_t)ww * n + j];
            pcb[k + 1 + j] = acc;
        }
        cluster.sync();  // 2
        // C
        T kl = T(0);
        for (int l = l0 + tid; l < nown; l += blockDim.x) {
            const int r = c + TD_CL * l;
            T acc = pvb[r];
            for (int cc = 0; cc < TD_CL; ++cc) acc += *cluster.map_shared_rank(pcb + r, cc);
            const T pr = beta * acc;
            pvb[r] = pr;
            kl = fma(pr, v[r - k - 1], kl);
        }
        block_sum(kl, b, 1);
        cluster.sync();  // 3
        // D
        cluster_sum(b, 1, 1);
        const T K = T(0.5) * beta * scal[1];
        for (int i = tid; i < m; i += blockDim.x) {
            const int r = k + 1 + i;
            w[i] = fma(-K, v[i], *cluster.map_shared_rank(pvb + r, r % TD_CL));
        }
        __syncthreads();
        for (int l = l0 + warp; l < nown; l += 8) {
            const int r = c + TD_CL * l, i = r - k - 1;
            T* row = L + off(l) + (k + 1);
            const T vi = v[i], wi = w[i];
            for (int j = lane; j <= i; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
        }
        if (c == 0 && tid == 0) t.e[k + 1] = alpha;
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            if (c == (n - 2) % TD_CL) t.d[n - 2] = L[off((n - 2 - c) / TD_CL) + (n - 2)];
            if (c == (n - 1) % TD_CL) {
                t.e[n - 1] = L[off((n - 1 - c) / TD_CL) + (n - 2)];
                t.d[n - 1] = L[off((n - 1 - c) / TD_CL) + (n - 1)];
            }
        } else if (n == 1 && c == 0) {
            t.d[0] = L[0];
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T>
bool launch_tridiag_dsm(const TridiagDescT<T>* d, int nmat, int maxn, cudaStream_t s) {
    const size_t smem = tridiag_dsm_smem<T>(maxn);
    if (smem > JAC_BLOCK_SMEM_MAX) return false;
    auto kern = tridiag_dsm_kernel<T>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nmat * TD_CL);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = TD_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        return false;
    }
    if (cudaLaunchKernelEx(&cfg, kern, d) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T>
void launch_tridiag(const TridiagDescT<T>* d, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    if (launch_tridiag_dsm<T>(d, nmat, maxn, s)) return;
    const size_t smem = 2 * (size_t)maxn * sizeof(T);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(tridiag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tridiag_kernel<T><<<nmat * JAC_CLUSTER, 256, smem, s>>>(d);
}
template void launch_tridiag<float>(const TridiagDescT<float>*, int, int, cudaStream_t);
template void launch_tridiag<double>(const TridiagDescT<double>*, int, int, cudaStream_t);

// All eigenvalues of symmetric tridiagonal matrices by bisection, one thread
// per eigenvalue j (ascending): eigenvalue j is the x where the Sturm count
// (number of eigenvalues below x = number of negative pivots of T - x I)
// passes j.  The count uses the leading principal minors
// p_i = (d_i - x) p_{i-1} - e_i^2 p_{i-2} (a pivot p_i / p_{i-1} is negative
// when consecutive minors differ in sign), which needs no division; minors are
// rescaled by powers of two to stay in range, and an exact zero minor is
// replaced by a tiny value of the opposite sign (the pivot counts as
// negative).  The interval starts from the Gershgorin bounds and is halved
// until it is no wider than 2 eps (|lo| + |hi|) or stops shrinking.
// Bit-level helpers of the Sturm count: sign, biased exponent and the range
// kept for the minors, per element type.
template <typename T>
struct SturmBits;
template <>
struct SturmBits<double> {
    using I = long long;
    static __device__ __forceinline__ I bits(double x) { return __double_as_longlong(x); }
    static __device__ __forceinline__ int expo(I b) { return (int)((b >> 52) & 0x7ff) - 1023; }
    static __device__ __forceinline__ bool is_zero(I b) { return (b & 0x7fffffffffffffffLL) == 0; }
    static constexpr int R = 400;
    static constexpr double up = 0x1p+400, down = 0x1p-400, tiny = 0x1p-1000;
    static constexpr double eps = 2.220446049250313e-16;
};
template <>
struct SturmBits<float> {
    using I = int;
    static __device__ __forceinline__ I bits(float x) { return __float_as_int(x); }
    static __device__ __forceinline__ int expo(I b) { return ((b >> 23) & 0xff) - 127; }
    static __device__ __forceinline__ bool is_zero(I b) { return (b & 0x7fffffff) == 0; }
    static constexpr int R = 40;
    static constexpr float up = 0x1p+40f, down = 0x1p-40f, tiny = 0x1p-120f;
    static constexpr float eps = 1.1920929e-07f;
};

template <typename T>
__device__ __forceinline__ int sturm_count(const T* __restrict__ d, const T* __restrict__ e2, int n, T x) {
    // signs and magnitudes are read from the bit patterns (integer pipe); the
    // floating-point work per step is one subtraction, one multiplication and
    // one FMA
    using B = SturmBits<T>;
    T p2 = T(1), p1 = d[0] - x;
    if (p1 == T(0)) p1 = -B::tiny;
    typename B::I b1 = B::bits(p1);
    int cnt = (b1 < 0);
    for (int i = 1; i < n; ++i) {
        T p = fma(d[i] - x, p1, -e2[i] * p2);
        typename B::I b = B::bits(p);
        if (B::is_zero(b)) {  // exact zero: opposite sign to p1, tiny magnitude
            p = (b1 < 0) ? B::tiny : -B::tiny;
            b = B::bits(p);
        }
        cnt += ((b ^ b1) < 0);
        const int ex = B::expo(b);
        if (ex > B::R) {
            p *= B::down;
            p1 *= B::down;
        } else if (ex < -B::R) {
            p *= B::up;
            p1 *= B::up;
        }
        p2 = p1;
        p1 = p;
        b1 = B::bits(p1);
    }
    return cnt;
}

template <typename T>
__global__ void __launch_bounds__(32) bisect_kernel(const TridiagDescT<T>* __restrict__ descs,
                                                     const int* __restrict__ eig_mat,
                                                     const int* __restrict__ eig_idx, int64_t total,
                                                     double* const* __restrict__ out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    const TridiagDescT<T> t = descs[eig_mat[gid]];
    const int j = eig_idx[gid];
    const int n = t.n;
    const T* e2 = t.e;  // squared in place by bisect_prepare_kernel
    T lo = T(0), hi = T(0);
    for (int i = 0; i < n; ++i) {
        const T r = (i > 0 ? sqrt(e2[i]) : T(0)) + (i + 1 < n ? sqrt(e2[i + 1]) : T(0));
        lo = (i == 0) ? t.d[i] - r : fmin(lo, t.d[i] - r);
        hi = (i == 0) ? t.d[i] + r : fmax(hi, t.d[i] + r);
    }
    const T eps = SturmBits<T>::eps;
    for (int it = 0; it < 200; ++it) {
        const T mid = T(0.5) * (lo + hi);
        if (!(mid > lo && mid < hi) || (hi - lo) <= T(2) * eps * (fabs(lo) + fabs(hi))) break;
        if (sturm_count<T>(t.d, e2, n, mid) > j)
            hi = mid;
        else
            lo = mid;
    }
    out[eig_mat[gid]][j] = (double)(T(0.5) * (lo + hi));
}

// e[i] <- e[i]^2 for every matrix (the bisection only needs the squares).
template <typename T>
__global__ void bisect_prepare_kernel(const TridiagDescT<T>* __restrict__ descs) {
    const TridiagDescT<T> t = descs[blockIdx.x];
    for (int i = threadIdx.x; i < t.n; i += blockDim.x) t.e[i] = t.e[i] * t.e[i];
}

template <typename T>
void launch_bisect(const TridiagDescT<T>* d, int nmat, const int* eig_mat, const int* eig_idx, int64_t total,
                   double* const* out, cudaStream_t s) {
    if (total <= 0) return;
    bisect_prepare_kernel<T><<<nmat, 256, 0, s>>>(d);
    // one warp per block so that the eigenvalues spread over every SM
    bisect_kernel<T><<<(unsigned)((total + 31) / 32), 32, 0, s>>>(d, eig_mat, eig_idx, total, out);
}
template void launch_bisect<float>(const TridiagDescT<float>*, int, const int*, const int*, int64_t, double* const*,
                                   cudaStream_t);
template void launch_bisect<double>(const TridiagDescT<double>*, int, const int*, const int*, int64_t,
                                    double* const*, cudaStream_t);

// ------------------------------------------------------------------ row GEMV
// One warp per output row, rows of all matrices in one flat list.
template <typename T>
__global__ void __launch_bounds__(256) gemv_rows_kernel(const GemvDescT<T>* __restrict__ descs,
                                                         const int* __restrict__ row_desc,
                                                         const int* __restrict__ row_local, int64_t nrows) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nrows) return;
    const GemvDescT<T> d = descs[row_desc[w]];
    const int r = row_local[w];
    int c0 = 0, c1 = d.ncols;
    if (d.mode == 1) c1 = min(r + 1, d.ncols);
    if (d.mode == 2) c0 = r;
    if (d.cstart) c0 = max(c0, d.cstart[r] - d.coff);
    if (d.cend) c1 = min(c1, d.cend[r] - d.coff);
    const T* row = d.M + (size_t)r * d.ld;
    T s0 = T(0), s1 = T(0);
    int c = c0 + lane;
    for (; c + 32 < c1; c += 64) {
        s0 = fma(row[c], d.x[c], s0);
        s1 = fma(row[c + 32], d.x[c + 32], s1);
    }
    if (c < c1) s0 = fma(row[c], d.x[c], s0);
    T s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d.y[r] = d.b ? fma(d.alpha, s, d.b[r]) : d.alpha * s;
}

template <typename T>
void launch_gemv_rows(const GemvDescT<T>* d, const int* row_desc, const int* row_local, int64_t nrows,
                      cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t threads = nrows * 32;
    const int64_t blocks = (threads + 255) / 256;
    gemv_rows_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d, row_desc, row_local, nrows);
}
template void launch_gemv_rows<float>(const GemvDescT<float>*, const int*, const int*, int64_t, cudaStream_t);
template void launch_gemv_rows<double>(const GemvDescT<double>*, const int*, const int*, int64_t, cudaStream_t);

// Local triangular products of the apply: one warp per group of RW
// consecutive rows of one matrix (mode 1: row r uses columns [0, r]; mode 2:
// [r, ncols)).  The descriptor is read once per group; each loop iteration
// issues 2 x RW independent coalesced row loads; x (one subdomain's vector)
// stays in L1.  Per row: lane-strided partial sums (two interleaved
// accumulators) and a fixed shuffle tree.
constexpr int GEMV_RW = GEMV_ROWS_PER_WARP;

template <typename T>
__global__ void __launch_bounds__(256) gemv_rows4_kernel(const GemvDescT<T>* __restrict__ descs,
                                                         const int* __restrict__ grp_desc,
                                                         const int* __restrict__ grp_row, int64_t ngroups) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ngroups) return;
    const GemvDescT<T> d = descs[grp_desc[w]];
    const int r0 = grp_row[w];
    const int nr = min(GEMV_RW, d.rows - r0);
    int lo[GEMV_RW], hi[GEMV_RW];
    int cmin = d.ncols, cmax = 0;
#pragma unroll
    for (int k = 0; k < GEMV_RW; ++k) {
        const int r = r0 + k;
        lo[k] = (d.mode == 2) ? r : 0;
        hi[k] = (d.mode == 1) ? min(r + 1, d.ncols) : d.ncols;
        if (k >= nr) hi[k] = lo[k];
        if (k < nr) {
            cmin = min(cmin, lo[k]);
            cmax = max(cmax, hi[k]);
        }
    }
    const T* M0 = d.M + (size_t)r0 * d.ld;
    T s[GEMV_RW], t[GEMV_RW];
#pragma unroll
    for (int k = 0; k < GEMV_RW; ++k) s[k] = t[k] = T(0);
    int c = cmin + lane;
    for (; c + 32 < cmax; c += 64) {
        const T x0 = d.x[c], x1 = d.x[c + 32];
#pragma unroll
        for (int k = 0; k < GEMV_RW; ++k) {
            if (c >= lo[k] && c < hi[k]) s[k] = fma(M0[(size_t)k * d.ld + c], x0, s[k]);
            if (c + 32 >= lo[k] && c + 32 < hi[k]) t[k] = fma(M0[(size_t)k * d.ld + c + 32], x1, t[k]);
        }
    }
    if (c < cmax) {
        const T x0 = d.x[c];
#pragma unroll
        for (int k = 0; k < GEMV_RW; ++k)
            if (c >= lo[k] && c < hi[k]) s[k] = fma(M0[(size_t)k * d.ld + c], x0, s[k]);
    }
    T mine = T(0);
#pragma unroll
    for (int k = 0; k < GEMV_RW; ++k) {
        T v = s[k] + t[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == k) mine = v;
    }
    if (lane < nr) {
        const int r = r0 + lane;
        d.y[r] = d.b ? fma(d.alpha, mine, d.b[r]) : d.alpha * mine;
    }
}

template <typename T>
void launch_gemv_rows4(const GemvDescT<T>* d, const int* grp_desc, const int* grp_row, int64_t ngroups,
                       cudaStream_t s) {
    if (ngroups <= 0) return;
    const int64_t blocks = (ngroups * 32 + 255) / 256;
    gemv_rows4_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d, grp_desc, grp_row, ngroups);
}
template void launch_gemv_rows4<float>(const GemvDescT<float>*, const int*, const int*, int64_t, cudaStream_t);
template void launch_gemv_rows4<double>(const GemvDescT<double>*, const int*, const int*, int64_t, cudaStream_t);

// The same products for nb <= MAXB right-hand sides (x_k = x + k xs, y_k = y
// + k ys; no b term): each factor entry is read once and applied to every
// x_k.  With GEMV_RW x MAXB = 32 the reduced sum of (row r, rhs k) is
// written by lane r MAXB + k.
template <typename T>
__global__ void __launch_bounds__(256) gemv_rows4_multi_kernel(const GemvDescT<T>* __restrict__ descs,
                                                               const int* __restrict__ grp_desc,
                                                               const int* __restrict__ grp_row, int64_t ngroups,
                                                               int nb, int64_t xs, int64_t ys) {
    static_assert(GEMV_RW * MAXB == 32, "one output per lane");
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ngroups) return;
    const GemvDescT<T> d = descs[grp_desc[w]];
    const int r0 = grp_row[w];
    const int nr = min(GEMV_RW, d.rows - r0);
    int lo[GEMV_RW], hi[GEMV_RW];
    int cmin = d.ncols, cmax = 0;
#pragma unroll
    for (int k = 0; k < GEMV_RW; ++k) {
        const int r = r0 + k;
        lo[k] = (d.mode == 2) ? r : 0;
        hi[k] = (d.mode == 1) ? min(r + 1, d.ncols) : d.ncols;
        if (k >= nr) hi[k] = lo[k];
        if (k < nr) {
            cmin = min(cmin, lo[k]);
            cmax = max(cmax, hi[k]);
        }
    }
    const T* M0 = d.M + (size_t)r0 * d.ld;
    T s[GEMV_RW][MAXB];
#pragma unroll
    for (int r = 0; r < GEMV_RW; ++r)
#pragma unroll
        for (int k = 0; k < MAXB; ++k) s[r][k] = T(0);
    for (int c = cmin + lane; c < cmax; c += 32) {
        T xv[MAXB];
#pragma unroll
        for (int k = 0; k < MAXB; ++k) xv[k] = k < nb ? d.x[k * xs + c] : T(0);
#pragma unroll
        for (int r = 0; r < GEMV_RW; ++r)
            if (c >= lo[r] && c < hi[r]) {
                const T m = M0[(size_t)r * d.ld + c];
#pragma unroll
                for (int k = 0; k < MAXB; ++k) s[r][k] = fma(m, xv[k], s[r][k]);
            }
    }
    T mine = T(0);
#pragma unroll
    for (int r = 0; r < GEMV_RW; ++r)
#pragma unroll
        for (int k = 0; k < MAXB; ++k) {
            T v = s[r][k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == r * MAXB + k) mine = v;
        }
    const int rr = lane / MAXB, kk = lane % MAXB;
    if (rr < nr && kk < nb) d.y[kk * ys + r0 + rr] = d.alpha * mine;
}

template <typename T>
void launch_gemv_rows4_multi(const GemvDescT<T>* d, const int* grp_desc, const int* grp_row, int64_t ngroups, int nb,
                             int64_t xs, int64_t ys, cudaStream_t s) {
    if (ngroups <= 0) return;
    const int64_t blocks = (ngroups * 32 + 255) / 256;
    gemv_rows4_multi_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d, grp_desc, grp_row, ngroups, nb, xs, ys);
}
template void launch_gemv_rows4_multi<float>(const GemvDescT<float>*, const int*, const int*, int64_t, int, int64_t,
                                             int64_t, cudaStream_t);
template void launch_gemv_rows4_multi<double>(const GemvDescT<double>*, const int*, const int*, int64_t, int, int64_t,
                                              int64_t, cudaStream_t);

// One warp per row of a batch of row-major matrices (mode 0: all columns),
// nb right-hand sides: y_k[row] = alpha (M x_k)[row].
template <typename T>
__global__ void __launch_bounds__(256) gemv_rows_multi_kernel(const GemvDescT<T>* __restrict__ descs,
                                                              const int* __restrict__ row_desc,
                                                              const int* __restrict__ row_local, int64_t nrows, int nb,
                                                              int64_t xs, int64_t ys) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nrows) return;
    const GemvDescT<T> d = descs[row_desc[w]];
    const int r = row_local[w];
    const T* row = d.M + (size_t)r * d.ld;
    T acc[MAXB];
#pragma unroll
    for (int k = 0; k < MAXB; ++k) acc[k] = T(0);
    for (int c = lane; c < d.ncols; c += 32) {
        const T m = row[c];
#pragma unroll
        for (int k = 0; k < MAXB; ++k)
            if (k < nb) acc[k] = fma(m, d.x[k * xs + c], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < MAXB; ++k) {
        T v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && k < nb) d.y[k * ys + r] = d.alpha * v;
    }
}

template <typename T>
void launch_gemv_rows_multi(const GemvDescT<T>* d, const int* row_desc, const int* row_local, int64_t nrows, int nb,
                            int64_t xs, int64_t ys, cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t blocks = (nrows * 32 + 255) / 256;
    gemv_rows_multi_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(d, row_desc, row_local, nrows, nb, xs, ys);
}
template void launch_gemv_rows_multi<double>(const GemvDescT<double>*, const int*, const int*, int64_t, int, int64_t,
                                             int64_t, cudaStream_t);

// ------------------------------------------------------------------ coarse solve
// L_E L_E^T e = c by blocked substitution in one cooperative launch.  The
// factor is split into K diagonal blocks of SB rows whose inverses Y_kk are
// stored.  Forward, for k = 0..K-1: y_k = Y_kk t_k (t = c, updated in
// place), then every later row r subtracts L[r, block k] y_k.  Backward, for
// k = K-1..0: e_k = Y_kk^T y_k, then every earlier row r subtracts
// (L^T)[r, block k] e_k.  Each phase spreads its rows over all warps of the
// grid (one warp per row, lane-strided products, fixed shuffle tree), and a
// grid-wide barrier separates the phases; rows outside the envelope of L_E
// (first column env_row[r], column r ends at env_colend[r]) are skipped.
// One CTA of 1024 threads per SM keeps the barrier to one arrival per SM.
// With nb right-hand sides (vectors ldv apart) each matrix entry is read once
// and applied to all of them.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int CSOLVE_THREADS = 1024;

// NB: the largest number of right-hand sides of the instantiation (1 for a
// single solve: no per-entry loop over right-hand sides at all).
template <int NB>
__global__ void __launch_bounds__(CSOLVE_THREADS) coarse_solve_kernel(CoarseSolveArgs a) {
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = a.n, SB = a.SB, K = a.K, nb = NB == 1 ? 1 : a.nb;
    const int64_t lv = a.ldv;
    double* t = a.c;
    double s[NB];
    auto reduce_store = [&](double* out, int idx, bool sub) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (k >= nb) break;
            const double v = warp_sum_d(s[k]);
            if (lane == 0) {
                if (sub)
                    out[k * lv + idx] -= v;
                else
                    out[k * lv + idx] = v;
            }
        }
    };
    for (int k0 = 0; k0 < K; ++k0) {
        const int r0 = k0 * SB, sb = min(SB, n - r0), r1 = r0 + sb;
        const double* Y = a.Yd + (size_t)k0 * SB * SB;
        for (int i = gw; i < sb; i += nw) {
            const double* row = Y + (size_t)i * SB;
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            for (int j = lane; j <= i; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, t[k * lv + r0 + j], s[k]);
            }
            reduce_store(a.y, r0 + i, false);
        }
        grid.sync();
        if (k0 + 1 == K) break;
        for (int r = r1 + gw; r < n; r += nw) {
            const int j0 = max(a.env_row[r], r0);
            if (j0 >= r1) continue;
            const double* row = a.L + (size_t)r * a.ld;
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            for (int j = j0 + lane; j < r1; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, a.y[k * lv + j], s[k]);
            }
            reduce_store(t, r, true);
        }
        grid.sync();
    }
    for (int k0 = K - 1; k0 >= 0; --k0) {
        const int r0 = k0 * SB, sb = min(SB, n - r0), r1 = r0 + sb;
        const double* Yt = a.Ydt + (size_t)k0 * SB * SB;
        for (int i = gw; i < sb; i += nw) {
            const double* row = Yt + (size_t)i * SB;
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            for (int j = i + lane; j < sb; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, a.y[k * lv + r0 + j], s[k]);
            }
            reduce_store(a.e, r0 + i, false);
        }
        if (k0 == 0) break;
        grid.sync();
        for (int r = gw; r < r0; r += nw) {
            const int j1 = min(a.env_colend[r], r1);
            if (j1 <= r0) continue;
            const double* row = a.Lt + (size_t)r * a.ld;
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            for (int j = r0 + lane; j < j1; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, a.e[k * lv + j], s[k]);
            }
            reduce_store(a.y, r, true);
        }
        grid.sync();
    }
}

template <int NB>
__global__ void __launch_bounds__(CSOLVE_THREADS) coarse_solve_folded_kernel(CoarseSolveArgs a) {
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = a.n, SB = a.SB, K = a.K, FW = a.FW, nb = NB == 1 ? 1 : a.nb;
    const int64_t lv = a.ldv;
    double s[NB];
    auto store = [&](double* out, int idx) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            if (k >= nb) break;
            const double v = warp_sum_d(s[k]);
            if (lane == 0) out[k * lv + idx] = v;
        }
    };
    // forward: y_k = Yd_k c_k - F_k y(window), windows of earlier blocks complete
    for (int k0 = 0; k0 < K; ++k0) {
        const int r0 = k0 * SB, sb = min(SB, n - r0);
        const double* Y = a.Yd + (size_t)k0 * SB * SB;
        const double* F = a.F + (size_t)k0 * SB * FW;
        const int w0 = a.fw0[k0], W = r0 - w0;
        for (int i = gw; i < sb; i += nw) {
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            const double* row = Y + (size_t)i * SB;
            for (int j = lane; j <= i; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, a.c[k * lv + r0 + j], s[k]);
            }
            const double* frow = F + (size_t)i * FW;
            for (int j = lane; j < W; j += 32) {
                const double m = frow[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(-m, a.y[k * lv + w0 + j], s[k]);
            }
            store(a.y, r0 + i);
        }
        grid.sync();
    }
    // backward: e_k = Ydt_k y_k - G_k e(window), windows of later blocks complete
    for (int k0 = K - 1; k0 >= 0; --k0) {
        const int r0 = k0 * SB, sb = min(SB, n - r0), r1 = r0 + sb;
        const double* Yt = a.Ydt + (size_t)k0 * SB * SB;
        const double* G = a.G + (size_t)k0 * SB * FW;
        const int V = a.gw1[k0] - r1;
        for (int i = gw; i < sb; i += nw) {
#pragma unroll
            for (int k = 0; k < NB; ++k) s[k] = 0.0;
            const double* row = Yt + (size_t)i * SB;
            for (int j = i + lane; j < sb; j += 32) {
                const double m = row[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(m, a.y[k * lv + r0 + j], s[k]);
            }
            const double* grow = G + (size_t)i * FW;
            for (int j = lane; j < V; j += 32) {
                const double m = grow[j];
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (NB == 1 || k < nb) s[k] = fma(-m, a.e[k * lv + r1 + j], s[k]);
            }
            store(a.e, r0 + i);
        }
        if (k0 > 0) grid.sync();
    }
}

int coarse_solve_blocks() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int per8 = 0;
    int pf = 0, pf8 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, coarse_solve_kernel<1>, CSOLVE_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per8, coarse_solve_kernel<MAXB>, CSOLVE_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, coarse_solve_folded_kernel<1>, CSOLVE_THREADS, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf8, coarse_solve_folded_kernel<MAXB>, CSOLVE_THREADS, 0) !=
            cudaSuccess)
        return 0;
    per = std::min(std::min(per, per8), std::min(pf, pf8));
    // one CTA per SM: the grid barriers between phases then take one arrival per SM
    return per >= 1 ? sms : 0;
}

cudaError_t launch_coarse_solve(const CoarseSolveArgs& a, int blocks, cudaStream_t s) {
    CoarseSolveArgs arg = a;
    void* params[] = {&arg};
    const void* fn = a.F ? (a.nb == 1 ? (const void*)coarse_solve_folded_kernel<1>
                                      : (const void*)coarse_solve_folded_kernel<MAXB>)
                         : (a.nb == 1 ? (const void*)coarse_solve_kernel<1> : (const void*)coarse_solve_kernel<MAXB>);
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(CSOLVE_THREADS), params, 0, s);
}

}  // namespace amdd
