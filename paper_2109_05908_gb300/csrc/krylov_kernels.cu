// Kernels of the deflated two-level preconditioner and of the one-level
// restricted additive Schwarz method (Sec. 4.1), and of right-preconditioned
// GMRES(m) (Saad and Schultz), the Krylov method the paper's experiments use
// with them (Sec. 4.1).
//
// Every reduction runs on a fixed grid (DOT_BLOCKS x 256) with fixed
// per-thread strides and fixed-order trees, so GMRES is bitwise reproducible
// for a given n.
#include "amdd_internal.h"

namespace amdd {

namespace {

__device__ __forceinline__ double bsum256(double v) {
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

inline unsigned grid_for(int64_t n, int64_t cap) {
    const int64_t want = (n + 255) / 256;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

// ------------------------------------------------------------------ RAS prolongation
// z[g] = yloc[own_idx[t]] (+ zc[t]) with g = order_g[t]: every unknown takes
// the local solution of the one subdomain whose Omega_Ii holds it (Boolean
// D_i), plus the coarse term in owner order.
template <typename TY>
__global__ void __launch_bounds__(256) ras_prolong_kernel(int64_t n, const int32_t* __restrict__ order_g,
                                                          const int32_t* __restrict__ own_idx,
                                                          const TY* __restrict__ yloc,
                                                          const double* __restrict__ zc, double* __restrict__ z) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double s = (double)yloc[own_idx[t]];
        if (zc) s += zc[t];
        z[order_g[t]] = s;
    }
}

template <typename TY>
void launch_ras_prolong(int64_t n, const int32_t* order_g, const int32_t* own_idx, const TY* yloc, const double* zc,
                        double* z, cudaStream_t s) {
    if (n <= 0) return;
    ras_prolong_kernel<TY><<<grid_for(n, 152 * 32), 256, 0, s>>>(n, order_g, own_idx, yloc, zc, z);
}
template void launch_ras_prolong<double>(int64_t, const int32_t*, const int32_t*, const double*, const double*,
                                         double*, cudaStream_t);
template void launch_ras_prolong<float>(int64_t, const int32_t*, const int32_t*, const float*, const double*, double*,
                                        cudaStream_t);

// zg[order_g[t]] = zo[t]: a vector in owner order to global order.
__global__ void __launch_bounds__(256) owner_to_global_kernel(int64_t n, const int32_t* __restrict__ order_g,
                                                              const double* __restrict__ zo,
                                                              double* __restrict__ zg) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        zg[order_g[t]] = zo[t];
}

void launch_owner_to_global(int64_t n, const int32_t* order_g, const double* zo, double* zg, cudaStream_t s) {
    if (n <= 0) return;
    owner_to_global_kernel<<<grid_for(n, 152 * 32), 256, 0, s>>>(n, order_g, zo, zg);
}

// out[t] = val[src[t]]
__global__ void __launch_bounds__(256) gather_idx64_kernel(const int64_t* __restrict__ src, int64_t cnt,
                                                           const double* __restrict__ val,
                                                           double* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = val[src[t]];
}

void launch_gather_idx64(const int64_t* src, int64_t cnt, const double* val, double* out, cudaStream_t s) {
    if (cnt > 0) gather_idx64_kernel<<<grid_for(cnt, 152 * 32), 256, 0, s>>>(src, cnt, val, out);
}

// ------------------------------------------------------------------ coarse ordering
__global__ void __launch_bounds__(256) sym_permute_kernel(const double* __restrict__ E, double* __restrict__ Ep,
                                                          const int32_t* __restrict__ perm, int64_t n) {
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t pr = perm[r];
        double* out = Ep + r * n;
        for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
            double v = 0.0;
            if (c <= r) {
                const int64_t pc = perm[c];
                v = pr >= pc ? E[pr * n + pc] : E[pc * n + pr];
            }
            out[c] = v;
        }
    }
}

void launch_sym_permute(const double* E, double* Ep, const int32_t* perm, int64_t n, cudaStream_t s) {
    if (n > 0) sym_permute_kernel<<<(unsigned)(n < 152 * 64 ? n : 152 * 64), 256, 0, s>>>(E, Ep, perm, n);
}

__global__ void __launch_bounds__(256) perm_move_kernel(int64_t n, const int32_t* __restrict__ perm,
                                                        const double* __restrict__ src, double* __restrict__ dst,
                                                        int nb, int64_t ld, int scatter) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = perm[r];
        for (int k = 0; k < nb; ++k) {
            if (scatter)
                dst[k * ld + q] = src[k * ld + r];
            else
                dst[k * ld + r] = src[k * ld + q];
        }
    }
}

void launch_perm_gather(int64_t n, const int32_t* perm, const double* src, double* dst, int nb, int64_t ld,
                        cudaStream_t s) {
    if (n > 0) perm_move_kernel<<<grid_for(n, 152 * 8), 256, 0, s>>>(n, perm, src, dst, nb, ld, 0);
}

void launch_perm_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, int nb, int64_t ld,
                         cudaStream_t s) {
    if (n > 0) perm_move_kernel<<<grid_for(n, 152 * 8), 256, 0, s>>>(n, perm, src, dst, nb, ld, 1);
}

// ------------------------------------------------------------------ residual SpMV
// y = b - A x, G lanes per row as in the plain SpMV.
template <int G>
__global__ void __launch_bounds__(256) spmv_resid_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ x, const double* __restrict__ b,
                                                         double* __restrict__ y) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (G - 1);
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t nround = ((n + groups - 1) / groups) * groups;
    for (int64_t row = gid / G; row < nround; row += groups) {
        double s = 0.0;
        if (row < n) {
            const int64_t lo = rowptr[row], hi = rowptr[row + 1];
            for (int64_t k = lo + sub; k < hi; k += G) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (row < n && sub == 0) y[row] = b[row] - s;
    }
}

void launch_spmv_resid(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                       const double* b, double* y, int group, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned blocks = grid_for(n * group, 152 * 64);
    if (group <= 1)
        spmv_resid_kernel<1><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, b, y);
    else if (group <= 4)
        spmv_resid_kernel<4><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, b, y);
    else if (group <= 8)
        spmv_resid_kernel<8><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, b, y);
    else
        spmv_resid_kernel<32><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, b, y);
}

// ------------------------------------------------------------------ GMRES(m)
// Classical Gram-Schmidt applied twice (CGS2) against the Arnoldi basis
// V_0..V_{k-1} (rows ldv apart, ldv even, 16-byte aligned), in three fused
// passes over the basis:
//   mode 0: partial sums of <V_j, w> for the KC vectors of chunk blockIdx.y;
//   mode 1: u = w - sum_j h_j V_j (written to out by chunk 0), partial sums of <V_j, u>;
//   mode 2: u = w - sum_j h_j V_j (written to out), partial sums of <u, u> (KC = 1).
// Each thread takes two consecutive elements per step (16-byte loads).
// Partial sums go to part[j * DOT_BLOCKS + blockIdx.x] (mode 2: part[blockIdx.x]).
template <int KC, int MODE>
__global__ void __launch_bounds__(256) gm_ortho_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int k,
                                                       const double* __restrict__ h, const double* __restrict__ w,
                                                       double* __restrict__ out, double* __restrict__ part) {
    __shared__ double hs[GM_MAXR + 1];
    __shared__ double wsum[8][KC];
    const int c0 = blockIdx.y * KC;
    const int kc = MODE == 2 ? 1 : min(KC, k - c0);
    if (MODE != 0)
        for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    double acc[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[j] = 0.0;
    const int64_t npair = n >> 1;
    for (int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x; q < npair; q += (int64_t)DOT_BLOCKS * 256) {
        const int64_t i = 2 * q;
        double2 u = *reinterpret_cast<const double2*>(w + i);
        if (MODE != 0) {
            double s0 = 0.0, s1 = 0.0;
            for (int j = 0; j < k; ++j) {
                // pass 2 reads each vector once (streaming); pass 1 reads its
                // block again for the dots below, so keeps it cached
                const double2* vp = reinterpret_cast<const double2*>(V + (int64_t)j * ldv + i);
                const double2 v = MODE == 2 ? __ldcs(vp) : *vp;
                s0 = fma(hs[j], v.x, s0);
                s1 = fma(hs[j], v.y, s1);
            }
            u.x -= s0;
            u.y -= s1;
            if (blockIdx.y == 0) *reinterpret_cast<double2*>(out + i) = u;
        }
        if (MODE == 2) {
            acc[0] = fma(u.x, u.x, acc[0]);
            acc[0] = fma(u.y, u.y, acc[0]);
        } else {
#pragma unroll
            for (int j = 0; j < KC; ++j)
                if (j < kc) {
                    const double2 v = *reinterpret_cast<const double2*>(V + (int64_t)(c0 + j) * ldv + i);
                    acc[j] = fma(v.x, u.x, acc[j]);
                    acc[j] = fma(v.y, u.y, acc[j]);
                }
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd n: the last element
        const int64_t i = n - 1;
        double u = w[i];
        if (MODE != 0) {
            double s0 = 0.0;
            for (int j = 0; j < k; ++j) s0 = fma(hs[j], V[(int64_t)j * ldv + i], s0);
            u -= s0;
            if (blockIdx.y == 0) out[i] = u;
        }
        if (MODE == 2) {
            acc[0] = fma(u, u, acc[0]);
        } else {
#pragma unroll
            for (int j = 0; j < KC; ++j)
                if (j < kc) acc[j] = fma(V[(int64_t)(c0 + j) * ldv + i], u, acc[j]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        if (j < kc) {
            double v = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wsum[warp][j] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < kc) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) v += wsum[q][threadIdx.x];
        part[(int64_t)(c0 + threadIdx.x) * DOT_BLOCKS + blockIdx.x] = v;
    }
}

void launch_gm_ortho(int64_t n, const double* V, int64_t ldv, int k, const double* h, const double* w, double* out,
                     double* part, int mode, cudaStream_t s) {
    if (mode == 0) {  // dots only: blocks of 8 vectors
        gm_ortho_kernel<8, 0><<<dim3(DOT_BLOCKS, (k + 7) / 8), 256, 0, s>>>(n, V, ldv, k, h, w, out, part);
    } else if (mode == 1) {  // update + dots: the update reads every vector, so one block row holds them all
        if (k <= 8)
            gm_ortho_kernel<8, 1><<<dim3(DOT_BLOCKS, 1), 256, 0, s>>>(n, V, ldv, k, h, w, out, part);
        else if (k <= 16)
            gm_ortho_kernel<16, 1><<<dim3(DOT_BLOCKS, 1), 256, 0, s>>>(n, V, ldv, k, h, w, out, part);
        else
            gm_ortho_kernel<GM_CHUNK, 1><<<dim3(DOT_BLOCKS, (k + GM_CHUNK - 1) / GM_CHUNK), 256, 0, s>>>(
                n, V, ldv, k, h, w, out, part);
    } else {
        gm_ortho_kernel<1, 2><<<dim3(DOT_BLOCKS, 1), 256, 0, s>>>(n, V, ldv, k, h, w, out, part);
    }
}

// hcol[j] = sum of the DOT_BLOCKS partial sums of vector j (fixed order);
// the Hessenberg column gets it (add = 0) or adds it (add = 1).
__global__ void __launch_bounds__(256) gm_finalize_kernel(const double* __restrict__ part, double* hcol, double* Hcol,
                                                          int add) {
    const int j = blockIdx.x;
    double v = 0.0;
    for (int t = threadIdx.x; t < DOT_BLOCKS; t += 256) v += part[(int64_t)j * DOT_BLOCKS + t];
    v = bsum256(v);
    if (threadIdx.x == 0) {
        hcol[j] = v;
        Hcol[j] = add ? Hcol[j] + v : v;
    }
}

void launch_gm_finalize(const double* part, int k, double* hcol, double* Hcol, int add, cudaStream_t s) {
    if (k > 0) gm_finalize_kernel<<<k, 256, 0, s>>>(part, hcol, Hcol, add);
}

// Norms: which 0 -> st->bnorm2 = ||b||^2; which 1 -> cycle start,
// beta = ||r||, g = beta e_1.
__global__ void __launch_bounds__(256) gm_norm_kernel(const double* __restrict__ part, GmState* st, int which) {
    double v = 0.0;
    for (int t = threadIdx.x; t < DOT_BLOCKS; t += 256) v += part[t];
    v = bsum256(v);
    if (threadIdx.x == 0) {
        if (which == 0) {
            st->bnorm2 = v;
        } else {
            st->beta = sqrt(v);
            st->g[0] = st->beta;
            for (int i = 1; i <= GM_MAXR; ++i) st->g[i] = 0.0;
        }
    }
}

void launch_gm_norm(const double* part, GmState* st, int which, cudaStream_t s) {
    gm_norm_kernel<<<1, 256, 0, s>>>(part, st, which);
}

// Arnoldi step j: h_{j+1,j} = ||u|| from the partial sums; the earlier
// Givens rotations applied to column j of H; a new rotation zeroing
// h_{j+1,j}; g updated; residual estimate |g_{j+1}| / ||b|| and the
// convergence flag.
__global__ void __launch_bounds__(256) gm_givens_kernel(const double* __restrict__ part, GmState* st, int j,
                                                        double rtol) {
    double v = 0.0;
    for (int t = threadIdx.x; t < DOT_BLOCKS; t += 256) v += part[t];
    v = bsum256(v);
    if (threadIdx.x == 0) {
        const double hn = sqrt(v);
        double* col = st->H + (int64_t)j * (GM_MAXR + 1);
        st->hnext = hn;
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = col[i], c = col[i + 1];
            col[i] = st->cs[i] * a + st->sn[i] * c;
            col[i + 1] = -st->sn[i] * a + st->cs[i] * c;
        }
        const double den = hypot(col[j], col[j + 1]);
        st->cs[j] = col[j] / den;
        st->sn[j] = col[j + 1] / den;
        col[j] = den;
        col[j + 1] = 0.0;
        st->g[j + 1] = -st->sn[j] * st->g[j];
        st->g[j] = st->cs[j] * st->g[j];
        const double bn = sqrt(st->bnorm2);
        st->res = fabs(st->g[j + 1]) / bn;
        st->conv = st->res <= rtol ? 1 : 0;
    }
}

void launch_gm_givens(const double* part, GmState* st, int j, double rtol, cudaStream_t s) {
    gm_givens_kernel<<<1, 256, 0, s>>>(part, st, j, rtol);
}

// dst = src / d with d = st->beta (which 0) or st->hnext (which 1); d = 0
// (exact breakdown) gives dst = 0.
__global__ void __launch_bounds__(256) gm_scale_kernel(int64_t n, const double* __restrict__ src, double* dst,
                                                       const GmState* __restrict__ st, int which) {
    const double d = which == 0 ? st->beta : st->hnext;
    const double f = d != 0.0 ? 1.0 / d : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = d != 0.0 ? src[i] * f : 0.0;
}

void launch_gm_scale(int64_t n, const double* src, double* dst, const GmState* st, int which, cudaStream_t s) {
    if (n > 0) gm_scale_kernel<<<grid_for(n, DOT_BLOCKS), 256, 0, s>>>(n, src, dst, st, which);
}

// y = H(0:k, 0:k)^{-1} g(0:k), back substitution on the rotated
// (upper-triangular) Hessenberg matrix; one thread (k <= GM_MAXR).
__global__ void gm_trisolve_kernel(GmState* st, int k) {
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int l = i + 1; l < k; ++l) s -= st->H[(int64_t)l * (GM_MAXR + 1) + i] * st->y[l];
        st->y[i] = s / st->H[(int64_t)i * (GM_MAXR + 1) + i];
    }
}

void launch_gm_trisolve(GmState* st, int k, cudaStream_t s) { gm_trisolve_kernel<<<1, 32, 0, s>>>(st, k); }

// x += sum_{j<k} y_j Zp_j (ascending j per element).
__global__ void __launch_bounds__(256) gm_combine_kernel(int64_t n, const double* __restrict__ Zp, int64_t ldv, int k,
                                                         const GmState* __restrict__ st, double* __restrict__ x) {
    __shared__ double ys[GM_MAXR];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = st->y[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(ys[j], Zp[(int64_t)j * ldv + i], s);
        x[i] += s;
    }
}

void launch_gm_combine(int64_t n, const double* Zp, int64_t ldv, int k, const GmState* st, double* x,
                       cudaStream_t s) {
    if (n > 0 && k > 0) gm_combine_kernel<<<grid_for(n, DOT_BLOCKS), 256, 0, s>>>(n, Zp, ldv, k, st, x);
}

}  // namespace amdd
