// Batched dense FP64 kernels for the subdomain blocks of the setup:
// tiled GEMM, blocked Cholesky (full or stopped early to leave a Schur
// complement), blocked inverse of the Cholesky factor, one-sided Jacobi row
// orthogonalisation (SVD of X_i, Sec. 3.2, and the symmetric eigensolve of
// eq. (Zi)), and small helpers.  One launch serves every subdomain at once
// (uneven sizes through per-matrix descriptors and flat tile lists).
#include <cooperative_groups.h>

#include "amdd_internal.h"

namespace cg = cooperative_groups;

namespace amdd {

// ------------------------------------------------------------------ GEMM
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs per thread, k
// staged through shared memory 16 at a time.  FP64 FMA throughout.
constexpr int GK = 16;

__global__ void __launch_bounds__(256) gemm_tiles_kernel(const GemmDesc* __restrict__ descs,
                                                          const TileRef* __restrict__ tiles, int ntiles) {
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const TileRef tr = tiles[t];
    const GemmDesc d = descs[tr.desc];
    __shared__ double As[GK][GEMM_T + 1];
    __shared__ double Bs[GK][GEMM_T + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = tr.tm * GEMM_T, col0 = tr.tn * GEMM_T;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    int kbeg = 0;
    if (d.kfrom_row) kbeg = (row0 / GK) * GK;
    for (int k0 = kbeg; k0 < d.k; k0 += GK) {
        for (int e = tid; e < GEMM_T * GK; e += 256) {
            int r, kk;
            if (!d.ta) { r = e / GK; kk = e % GK; } else { kk = e / GEMM_T; r = e % GEMM_T; }
            const int gr = row0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gr < d.m && gk < d.k)
                v = d.ta ? d.A[(size_t)gk * d.lda + gr] : d.A[(size_t)gr * d.lda + gk];
            As[kk][r] = v;
        }
        for (int e = tid; e < GEMM_T * GK; e += 256) {
            int c, kk;
            if (!d.tb) { kk = e / GEMM_T; c = e % GEMM_T; } else { c = e / GK; kk = e % GK; }
            const int gc = col0 + c, gk = k0 + kk;
            double v = 0.0;
            if (gc < d.n && gk < d.k)
                v = d.tb ? d.B[(size_t)gc * d.ldb + gk] : d.B[(size_t)gk * d.ldb + gc];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= d.m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx + 16 * j;
            if (c >= d.n || (d.lower && c > r)) continue;
            double* cp = d.C + (size_t)r * d.ldc + c;
            const double v = d.alpha * acc[i][j];
            *cp = (d.beta != 0.0) ? fma(d.beta, *cp, v) : v;
        }
    }
}

void launch_gemm(const GemmDesc* d_descs, const TileRef* d_tiles, int ntiles, cudaStream_t s) {
    if (ntiles > 0) gemm_tiles_kernel<<<ntiles, 256, 0, s>>>(d_descs, d_tiles, ntiles);
}

// ------------------------------------------------------------------ Cholesky
// Factor the NB x NB diagonal block [k0, k0+kb) of each matrix in shared
// memory (its trailing part already updated by earlier steps), write L back
// and store the inverse of the block for the panel solve and for the inverse
// factor.  With a pivot floor (clamp) a pivot below it is raised to it;
// without, a pivot <= 0 (or NaN) latches DERR_NOT_SPD and is replaced by 1 so
// the factorisation finishes with finite numbers.
__global__ void __launch_bounds__(256) chol_diag_kernel(const CholDesc* __restrict__ descs, int k0,
                                                         int* __restrict__ err) {
    const CholDesc d = descs[blockIdx.x];
    const int kend = min(k0 + CHOL_NB, d.stop);
    if (k0 >= kend) return;
    const int kb = kend - k0;
    __shared__ double L[CHOL_NB][CHOL_NB + 1];
    __shared__ double Li[CHOL_NB][CHOL_NB + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += blockDim.x) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        L[r][c] = (r < kb && c <= r) ? d.A[(size_t)(k0 + r) * d.ld + (k0 + c)] : 0.0;
        Li[r][c] = 0.0;
    }
    __syncthreads();
    const double floor_v = d.clamp ? *d.clamp : 0.0;
    for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
            double piv = L[j][j];
            if (d.clamp) {
                if (!(piv >= floor_v)) piv = floor_v;
            } else if (!(piv > 0.0)) {
                atomicOr(err, DERR_NOT_SPD);
                piv = 1.0;
            }
            L[j][j] = sqrt(piv);
        }
        __syncthreads();
        if (tid > j && tid < kb) L[tid][j] /= L[j][j];
        __syncthreads();
        for (int e = tid; e < CHOL_NB * CHOL_NB; e += blockDim.x) {
            const int r = e / CHOL_NB, c = e % CHOL_NB;
            if (c > j && r >= c && r < kb) L[r][c] = fma(-L[r][j], L[c][j], L[r][c]);
        }
        __syncthreads();
    }
    // inverse of the lower-triangular block, one column per thread
    if (tid < kb) {
        const int c = tid;
        for (int r = c; r < kb; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) s = fma(-L[r][k], Li[k][c], s);
            Li[r][c] = s / L[r][r];
        }
    }
    __syncthreads();
    double* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += blockDim.x) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        if (r < kb && c <= r) d.A[(size_t)(k0 + r) * d.ld + (k0 + c)] = L[r][c];
        linv[e] = (r < kb && c < kb) ? Li[r][c] : 0.0;
    }
}

void launch_chol_diag(const CholDesc* d, int nmat, int k0, int* err, cudaStream_t s) {
    if (nmat > 0) chol_diag_kernel<<<nmat, 256, 0, s>>>(d, k0, err);
}

// Panel below the diagonal block: A[r, k0:k0+kb] <- A[r, k0:k0+kb] * Linv^T
// for 64 rows per CTA.
__global__ void __launch_bounds__(256) chol_panel_kernel(const CholDesc* __restrict__ descs,
                                                          const PanelRef* __restrict__ tiles, int k0) {
    const PanelRef t = tiles[blockIdx.x];
    const CholDesc d = descs[t.desc];
    const int kend = min(k0 + CHOL_NB, d.stop);
    const int kb = kend - k0;
    const int r0 = kend + t.rt * 64;
    __shared__ double Li[CHOL_NB][CHOL_NB + 1];
    __shared__ double P[64][CHOL_NB + 1];
    const double* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += 256) Li[e / CHOL_NB][e % CHOL_NB] = linv[e];
    for (int e = tid; e < 64 * CHOL_NB; e += 256) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        const int gr = r0 + r;
        P[r][c] = (gr < d.n && c < kb) ? d.A[(size_t)gr * d.ld + (k0 + c)] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < 64 * CHOL_NB; e += 256) {
        const int r = e / CHOL_NB, c = e % CHOL_NB;
        const int gr = r0 + r;
        if (c < kb && gr < d.n) {
            double s = 0.0;
            for (int k = 0; k <= c; ++k) s = fma(P[r][k], Li[c][k], s);
            d.A[(size_t)gr * d.ld + (k0 + c)] = s;
        }
    }
}

void launch_chol_panel(const CholDesc* d, const PanelRef* tiles, int ntiles, int k0, cudaStream_t s) {
    if (ntiles > 0) chol_panel_kernel<<<ntiles, 256, 0, s>>>(d, tiles, k0);
}

// ------------------------------------------------------------------ inverse factor
// Y = L^{-1} by blocked forward substitution on the identity: for each
// diagonal block k, Y[k-rows, 0:kend] <- Linv_k * Y[k-rows, 0:kend]; the
// trailing update Y[kend:, 0:kend] -= L[kend:, k-cols] * Y[k-rows, 0:kend]
// is a GEMM issued by the host.
__global__ void __launch_bounds__(256) trtri_diag_kernel(const TrtriDesc* __restrict__ descs,
                                                          const ChunkRef* __restrict__ tiles, int k0) {
    const ChunkRef t = tiles[blockIdx.x];
    const TrtriDesc d = descs[t.desc];
    const int kend = min(k0 + CHOL_NB, d.n);
    const int kb = kend - k0;
    const int c0 = t.ct * 64;
    __shared__ double Li[CHOL_NB][CHOL_NB + 1];
    __shared__ double B[CHOL_NB][64 + 1];
    const double* linv = d.Linv + (size_t)(k0 / CHOL_NB) * CHOL_NB * CHOL_NB;
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_NB * CHOL_NB; e += 256) Li[e / CHOL_NB][e % CHOL_NB] = linv[e];
    for (int e = tid; e < CHOL_NB * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        B[r][c] = (r < kb && c0 + c < kend) ? d.Y[(size_t)(k0 + r) * d.ldy + (c0 + c)] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < CHOL_NB * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        if (r < kb && c0 + c < kend) {
            double s = 0.0;
            for (int k = 0; k <= r; ++k) s = fma(Li[r][k], B[k][c], s);
            d.Y[(size_t)(k0 + r) * d.ldy + (c0 + c)] = s;
        }
    }
}

void launch_trtri_diag(const TrtriDesc* d, const ChunkRef* tiles, int ntiles, int k0, cudaStream_t s) {
    if (ntiles > 0) trtri_diag_kernel<<<ntiles, 256, 0, s>>>(d, tiles, k0);
}

__global__ void set_identity_kernel(const TrtriDesc* __restrict__ descs) {
    const TrtriDesc d = descs[blockIdx.y];
    for (int r = blockIdx.x; r < d.n; r += gridDim.x) {
        double* row = d.Y + (size_t)r * d.ldy;
        for (int c = threadIdx.x; c < d.n; c += blockDim.x) row[c] = (r == c) ? 1.0 : 0.0;
    }
}

void launch_set_identity(const TrtriDesc* d, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid(min(maxn, 1024), nmat);
    set_identity_kernel<<<grid, 256, 0, s>>>(d);
}

// ------------------------------------------------------------------ Jacobi
// One-sided (Hestenes) Jacobi on the rows of each matrix, in T = float or
// double: rotate row pairs until every pair is orthogonal over the first
// ncols_dot columns to tol relative to the row norms (and, when a floor is
// given, above that absolute floor on |<p,q>|); rotations are applied to
// ncols_rot columns (so an identity appended on the right accumulates them).
// Row norms^2 are recomputed at the start of each sweep and updated exactly
// after each rotation (a' = a - t g, b' = b + t g), so a pair that needs no
// rotation costs one inner product.  A cluster of JAC_CLUSTER CTAs works on
// one matrix; each round of the round-robin (circle) schedule holds rows/2
// disjoint pairs, one warp per pair, and the cluster barrier separates
// rounds.  Every thread of the cluster runs the same number of barriers: the
// sweep loop ends on a value all threads compute identically from the CTAs'
// shared flags (read through distributed shared memory), and is bounded by
// max_sweeps.
template <typename T>
__device__ __forceinline__ T ldcg_t(const T* p) {
    return __ldcg(p);
}

template <typename T>
__global__ void __cluster_dims__(JAC_CLUSTER, 1, 1) __launch_bounds__(256)
    jacobi_rows_kernel(const JacobiDescT<T>* __restrict__ descs, int max_sweeps, T tol, int* __restrict__ sweeps,
                       unsigned long long* __restrict__ rots, int* __restrict__ err, int report_noconv) {
    cg::cluster_group cluster = cg::this_cluster();
    const int mat = blockIdx.x / JAC_CLUSTER;
    const int crank = (int)cluster.block_rank();
    const JacobiDescT<T> d = descs[mat];
    __shared__ int rotated;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    const int gw = crank * wpc + warp, nw = JAC_CLUSTER * wpc;
    const int m = d.rows + (d.rows & 1);
    const int npairs = m / 2;
    const int nrounds = m - 1;
    const T absf = d.absfloor ? *d.absfloor : T(0);
    int sweep = 0;
    bool done = false;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        // row norms^2 at the start of the sweep
        for (int r = gw; r < d.rows; r += nw) {
            const T* x = d.A + (size_t)r * d.ld;
            T a = T(0);
            for (int c = lane; c < d.ncols_dot; c += 32) {
                const T u = ldcg_t(x + c);
                a = fma(u, u, a);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) d.nrm2[r] = a;
        }
        __threadfence();
        cluster.sync();
        for (int r = 0; r < nrounds; ++r) {
            for (int k = gw; k < npairs; k += nw) {
                int p, q;
                if (k == 0) {
                    p = m - 1;
                    q = r;
                } else {
                    p = (r + k) % (m - 1);
                    q = (r - k + (m - 1)) % (m - 1);
                }
                if (p >= d.rows || q >= d.rows) continue;
                T* xp = d.A + (size_t)p * d.ld;
                T* xq = d.A + (size_t)q * d.ld;
                T g = T(0);
                for (int c = lane; c < d.ncols_dot; c += 32) g = fma(ldcg_t(xp + c), ldcg_t(xq + c), g);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                const T a = ldcg_t(d.nrm2 + p), b = ldcg_t(d.nrm2 + q);
                if (g != T(0) && fabs(g) > tol * sqrt(a) * sqrt(b) && fabs(g) > absf) {
                    const T zeta = (b - a) / (T(2) * g);
                    const T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
                    const T cs = T(1) / sqrt(fma(t, t, T(1)));
                    const T sn = cs * t;
                    for (int c = lane; c < d.ncols_rot; c += 32) {
                        const T u = ldcg_t(xp + c), v = ldcg_t(xq + c);
                        xp[c] = fma(cs, u, -sn * v);
                        xq[c] = fma(sn, u, cs * v);
                    }
                    if (lane == 0) {
                        d.nrm2[p] = fma(-t, g, a);
                        d.nrm2[q] = fma(t, g, b);
                        rotated = 1;
                        atomicAdd(rots + mat, 1ull);
                    }
                }
            }
            __threadfence();
            cluster.sync();
        }
        int any = 0;
#pragma unroll
        for (int rr = 0; rr < JAC_CLUSTER; ++rr) any |= *cluster.map_shared_rank(&rotated, rr);
        cluster.sync();
        if (!any) {
            done = true;
            break;
        }
    }
    if (crank == 0 && threadIdx.x == 0) {
        sweeps[mat] = done ? sweep + 1 : sweep;
        if (!done && report_noconv) atomicOr(err, DERR_EIG_NOCONV);
    }
}

template <typename T>
void launch_jacobi_t(const JacobiDescT<T>* d, int nmat, int max_sweeps, T tol, int* sweeps, unsigned long long* rots,
                     int* err, int report_noconv, cudaStream_t s) {
    if (nmat > 0)
        jacobi_rows_kernel<T><<<nmat * JAC_CLUSTER, 256, 0, s>>>(d, max_sweeps, tol, sweeps, rots, err, report_noconv);
}
template void launch_jacobi_t<float>(const JacobiDescT<float>*, int, int, float, int*, unsigned long long*, int*, int,
                                     cudaStream_t);
template void launch_jacobi_t<double>(const JacobiDescT<double>*, int, int, double, int*, unsigned long long*, int*,
                                      int, cudaStream_t);

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

// Row norms over ncols_dot, delta = eps * max norm, optional row scaling by
// 1/sqrt(norm) over ncols_rot.  One CTA per matrix, one warp per row.
__global__ void __launch_bounds__(256) rownorms_kernel(const JacobiDesc* __restrict__ descs,
                                                        double* const* __restrict__ sig, double* __restrict__ delta,
                                                        double eps, int scale_rows) {
    const JacobiDesc d = descs[blockIdx.x];
    double* out = sig[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double wmax[8];
    double mx = 0.0;
    for (int r = warp; r < d.rows; r += 8) {
        double* row = d.A + (size_t)r * d.ld;
        double s = 0.0;
        for (int c = lane; c < d.ncols_dot; c += 32) s = fma(row[c], row[c], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double nrm = sqrt(s);
        if (lane == 0) out[r] = nrm;
        mx = fmax(mx, nrm);
        if (scale_rows && nrm > 0.0) {
            const double f = 1.0 / sqrt(nrm);
            for (int c = lane; c < d.ncols_rot; c += 32) row[c] *= f;
        }
    }
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < 8; ++w) m = fmax(m, wmax[w]);
        if (delta) delta[blockIdx.x] = eps * m;
    }
}

void launch_rownorms(const JacobiDesc* d, int nmat, double* const* sigma_ptrs, double* delta, double eps,
                     int scale_rows, cudaStream_t s) {
    if (nmat > 0) rownorms_kernel<<<nmat, 256, 0, s>>>(d, sigma_ptrs, delta, eps, scale_rows);
}

__global__ void add_diag_kernel(double* const* __restrict__ mats, const int* __restrict__ n,
                                const int* __restrict__ ld, const double* __restrict__ delta) {
    const int b = blockIdx.y;
    double* M = mats[b];
    const double dv = delta[b];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n[b]; j += gridDim.x * blockDim.x)
        M[(size_t)j * ld[b] + j] += dv;
}

void launch_add_diag(double* const* mats, const int* n, const int* ld, const double* delta, int nmat, int maxn,
                     cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid((maxn + 255) / 256, nmat);
    add_diag_kernel<<<grid, 256, 0, s>>>(mats, n, ld, delta);
}

__global__ void mirror_lower_kernel(double* const* __restrict__ mats, const int* __restrict__ n,
                                    const int* __restrict__ ld) {
    const int b = blockIdx.y;
    double* M = mats[b];
    const int nn = n[b], l = ld[b];
    for (int r = blockIdx.x; r < nn; r += gridDim.x)
        for (int c = r + 1 + threadIdx.x; c < nn; c += blockDim.x) M[(size_t)r * l + c] = M[(size_t)c * l + r];
}

void launch_mirror_lower(double* const* mats, const int* n, const int* ld, int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    dim3 grid(min(maxn, 1024), nmat);
    mirror_lower_kernel<<<grid, 128, 0, s>>>(mats, n, ld);
}

// dst = src^T for square n x n matrices, 32 x 32 tiles through shared memory.
__global__ void transpose_kernel(const double* const* __restrict__ src, double* const* __restrict__ dst,
                                 const int* __restrict__ n, const int* __restrict__ lds,
                                 const int* __restrict__ ldd) {
    const int b = blockIdx.z;
    const int nn = n[b];
    const int nt = (nn + 31) / 32;
    __shared__ double tile[32][33];
    for (int t = blockIdx.x; t < nt * nt; t += gridDim.x) {
        const int tr = t / nt, tc = t % nt;
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int r = e / 32, c = e % 32;
            const int gr = tr * 32 + r, gc = tc * 32 + c;
            tile[r][c] = (gr < nn && gc < nn) ? src[b][(size_t)gr * lds[b] + gc] : 0.0;
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

void launch_transpose(const double* const* src, double* const* dst, const int* n, const int* lds, const int* ldd,
                      int nmat, int maxn, cudaStream_t s) {
    if (nmat <= 0 || maxn <= 0) return;
    const int nt = (maxn + 31) / 32;
    dim3 grid(min(nt * nt, 4096), 1, nmat);
    transpose_kernel<<<grid, 256, 0, s>>>(src, dst, n, lds, ldd);
}

// ------------------------------------------------------------------ row GEMV
// One warp per output row, rows of all matrices in one flat list.
__global__ void __launch_bounds__(256) gemv_rows_kernel(const GemvDesc* __restrict__ descs,
                                                         const int* __restrict__ row_desc,
                                                         const int* __restrict__ row_local, int64_t nrows) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nrows) return;
    const GemvDesc d = descs[row_desc[w]];
    const int r = row_local[w];
    int c0 = 0, c1 = d.ncols;
    if (d.mode == 1) c1 = min(r + 1, d.ncols);
    if (d.mode == 2) c0 = r;
    const double* row = d.M + (size_t)r * d.ld;
    double s = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) s = fma(row[c], d.x[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d.y[r] = s;
}

void launch_gemv_rows(const GemvDesc* d, const int* row_desc, const int* row_local, int64_t nrows, cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t threads = nrows * 32;
    const int64_t blocks = (threads + 255) / 256;
    gemv_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, row_desc, row_local, nrows);
}

}  // namespace amdd
