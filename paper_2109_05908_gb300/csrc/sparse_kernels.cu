// Sparse and vector kernels: CSR SpMV (Sec. 1, the operator of A x = b),
// restriction / prolongation of the additive Schwarz apply
// (Eq. (two_level_schwarz)), coarse-matrix blocks E_ij = Z_i^T A_{I_i I_j} Z_j,
// and the deterministic reductions and updates of PCG.
#include "amdd_internal.h"

namespace amdd {

// ------------------------------------------------------------------ SpMV
// G lanes per row (G in {1, 8, 32}); rows are assigned to lane groups in a
// grid-stride loop.  G = 1 (rows of at most 8 entries): the entries of a
// row load in parallel and a warp covers 32 consecutive rows.
template <int G>
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                                   const double* __restrict__ x, double* __restrict__ y) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = threadIdx.x & (G - 1);
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    // every lane of the grid runs the same number of iterations, so the full
    // warp takes part in each shuffle
    const int64_t nround = ((n + groups - 1) / groups) * groups;
    for (int64_t row = gid / G; row < nround; row += groups) {
        double s = 0.0;
        if (row < n) {
            const int64_t b = rowptr[row], e = rowptr[row + 1];
            for (int64_t k = b + sub; k < e; k += G) s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (row < n && sub == 0) y[row] = s;
    }
}

int spmv_group_for(int64_t n, int64_t nnz) {
    const int64_t per = n > 0 ? nnz / n : 0;
    return per <= 8 ? 1 : (per <= 24 ? 8 : 32);
}

void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y, int group, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t want = (n * group + 255) / 256;
    const int blocks = (int)(want < 152 * 64 ? want : 152 * 64);
    if (group <= 1)
        spmv_kernel<1><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
    else if (group <= 4)
        spmv_kernel<4><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
    else if (group <= 8)
        spmv_kernel<8><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
    else
        spmv_kernel<32><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
}

// y_k = A x_k for nb <= MAXB right-hand sides stored ld apart: one thread per
// row reads the row's entries once and applies them to every x_k.
__global__ void __launch_bounds__(256) spmv_multi_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val, const double* __restrict__ x,
                                                         double* __restrict__ y, int nb, int64_t ld) {
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        double acc[MAXB];
#pragma unroll
        for (int k = 0; k < MAXB; ++k) acc[k] = 0.0;
        for (int64_t e = rowptr[row]; e < rowptr[row + 1]; ++e) {
            const double v = __ldg(val + e);
            const int64_t c = __ldg(col + e);
#pragma unroll
            for (int k = 0; k < MAXB; ++k)
                if (k < nb) acc[k] = fma(v, __ldg(x + k * ld + c), acc[k]);
        }
#pragma unroll
        for (int k = 0; k < MAXB; ++k)
            if (k < nb) y[k * ld + row] = acc[k];
    }
}

void launch_spmv_multi(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                       double* y, int nb, int64_t ld, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t want = (n + 255) / 256;
    spmv_multi_kernel<<<(unsigned)(want < 152 * 64 ? want : 152 * 64), 256, 0, s>>>(n, rowptr, col, val, x, y, nb, ld);
}

// ------------------------------------------------------------------ sparse local factors
// dst[t] = src[idx[t]] for idx[t] >= 0, and 1 / src[-idx[t] - 1] otherwise
// (the diagonal of a factor column is stored as its reciprocal)
template <typename T>
__global__ void gather_entries_kernel(const T* __restrict__ src, const int64_t* __restrict__ idx,
                                      T* __restrict__ dst, int64_t cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx[t];
        dst[t] = k >= 0 ? src[k] : T(1) / src[-k - 1];
    }
}

template <typename T>
void launch_gather_entries(const T* src, const int64_t* idx, T* dst, int64_t cnt, cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t want = (cnt + 255) / 256;
    gather_entries_kernel<T><<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(src, idx, dst, cnt);
}
template void launch_gather_entries<float>(const float*, const int64_t*, float*, int64_t, cudaStream_t);
template void launch_gather_entries<double>(const double*, const int64_t*, double*, int64_t, cudaStream_t);

// The local solves of the Schwarz methods with sparse Cholesky factors in a
// nested-dissection order: y_i = P^T L^{-T} L^{-1} P r_i for every subdomain,
// one warp (one CTA) per subdomain and up to 8 right-hand sides at once.  The
// factor's columns (CSC, the diagonal first and stored as its reciprocal,
// 16-bit row indices) and the nb vectors are staged in shared memory; the warp
// splits into nb groups of gs lanes (gs = 32 / nb rounded down to a power of
// two), group v working on vector v:
//   forward  (column j ascending):  w_j = x_j / l_jj,  x_i -= l_ij w_j (i > j);
//   backward (column j descending): z_j = (w_j - sum_{i>j} l_ij z_i) / l_jj,
// the sum lane-strided over the column's entries with a fixed shuffle tree
// inside the group, so the result is reproducible run to run.  r and y hold nb
// vectors, ld apart.
template <typename T>
__global__ void __launch_bounds__(32) sparse_local_solve_kernel(const SparseLocalDesc* __restrict__ descs,
                                                                const int32_t* __restrict__ colptr,
                                                                const uint16_t* __restrict__ rowidx,
                                                                const T* __restrict__ val,
                                                                const int32_t* __restrict__ perm,
                                                                const T* __restrict__ r, T* __restrict__ y, int nb,
                                                                int64_t ld) {
    extern __shared__ __align__(16) unsigned char sl_raw[];
    const SparseLocalDesc d = descs[blockIdx.x];
    const int n = d.n, lane = threadIdx.x;
    const int nnz = d.nnz;
    T* v = reinterpret_cast<T*>(sl_raw);
    T* x = v + nnz;  // nb vectors of n
    int32_t* cp = reinterpret_cast<int32_t*>(x + (size_t)nb * n);
    uint16_t* rw = reinterpret_cast<uint16_t*>(cp + n + 1);
    const int32_t* gcp = colptr + d.poff;
    for (int k = lane; k <= n; k += 32) cp[k] = gcp[k];
    for (int k = lane; k < nnz; k += 32) {
        v[k] = val[d.eoff + k];
        rw[k] = rowidx[d.eoff + k];
    }
    const int32_t* pm = perm + d.xoff;
    for (int e = lane; e < nb * n; e += 32) {
        const int vec = e / n, a = e - vec * n;
        x[e] = r[(size_t)vec * ld + d.xoff + pm[a]];
    }
    int gs = 32;
    while (gs > 1 && gs * nb > 32) gs >>= 1;
    const int vec = lane / gs, sub = lane % gs;
    const bool act = vec < nb;
    T* xv = x + (size_t)(act ? vec : 0) * n;
    __syncwarp();
    // forward: column j reads x_j (final once the earlier columns are done) and
    // updates rows > j only, so x_j itself is scaled by 1 / l_jj in one pass
    // after the loop
    for (int j = 0; j < n; ++j) {
        const int b = cp[j], e = cp[j + 1];
        if (act) {
            const T wj = xv[j] * v[b];
            for (int k = b + 1 + sub; k < e; k += gs) xv[rw[k]] = fma(-v[k], wj, xv[rw[k]]);
        }
        __syncwarp();
    }
    for (int e = lane; e < nb * n; e += 32) {
        const int a = e % n;
        x[e] *= v[cp[a]];
    }
    __syncwarp();
    for (int j = n - 1; j >= 0; --j) {
        const int b = cp[j], e = cp[j + 1];
        T sum = T(0);
        if (act)
            for (int k = b + 1 + sub; k < e; k += gs) sum = fma(v[k], xv[rw[k]], sum);
        for (int o = gs / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (act && sub == 0) xv[j] = (xv[j] - sum) * v[b];
        __syncwarp();
    }
    for (int e = lane; e < nb * n; e += 32) {
        const int vv = e / n, a = e - vv * n;
        y[(size_t)vv * ld + d.xoff + pm[a]] = x[e];
    }
}

template <typename T>
size_t sparse_local_smem(int n, int nnz, int nb) {
    return (size_t)((size_t)nb * n + nnz) * sizeof(T) + (size_t)(n + 1) * sizeof(int32_t) +
           (size_t)nnz * sizeof(uint16_t) + 16;
}
template size_t sparse_local_smem<float>(int, int, int);
template size_t sparse_local_smem<double>(int, int, int);

template <typename T>
void launch_sparse_local_solve(const SparseLocalDesc* d, int nmat, size_t smem, const int32_t* colptr,
                               const uint16_t* rowidx, const T* val, const int32_t* perm, const T* r, T* y, int nb,
                               int64_t ld, cudaStream_t s) {
    if (nmat <= 0) return;
    cudaFuncSetAttribute(sparse_local_solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sparse_local_solve_kernel<T><<<nmat, 32, smem, s>>>(d, colptr, rowidx, val, perm, r, y, nb, ld);
}
template void launch_sparse_local_solve<float>(const SparseLocalDesc*, int, size_t, const int32_t*, const uint16_t*,
                                               const float*, const int32_t*, const float*, float*, int, int64_t,
                                               cudaStream_t);
template void launch_sparse_local_solve<double>(const SparseLocalDesc*, int, size_t, const int32_t*,
                                                const uint16_t*, const double*, const int32_t*, const double*,
                                                double*, int, int64_t, cudaStream_t);

// ------------------------------------------------------------------ input checks
// *flag |= 1 if any of v[0..n) is NaN or infinite (the flag is only ever set)
__global__ void nonfinite_kernel(const double* __restrict__ v, int64_t n, int* __restrict__ flag) {
    bool bad = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(__ldg(v + t));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_nonfinite(const double* v, int64_t n, int* flag, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t want = (n + 255) / 256;
    nonfinite_kernel<<<(unsigned)(want < 152 * 16 ? want : 152 * 16), 256, 0, s>>>(v, n, flag);
}

// ------------------------------------------------------------------ gathers
__global__ void gather_values_kernel(const int64_t* __restrict__ src, const int64_t* __restrict__ dst, int64_t cnt,
                                     const double* __restrict__ val, double* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        out[dst[t]] = val[src[t]];
}

void launch_gather_values(const int64_t* src, const int64_t* dst, int64_t cnt, const double* val, double* out,
                          cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t want = (cnt + 255) / 256;
    gather_values_kernel<<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(src, dst, cnt, val, out);
}

__global__ void gather_vec_kernel(const int32_t* __restrict__ idx, int64_t cnt, const double* __restrict__ x,
                                  double* __restrict__ out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = x[idx[t]];
}

// out[k][t] = x[k][idx[t]] for nb right-hand sides (x stride ldx, out stride cnt)
__global__ void gather_vec_multi_kernel(const int32_t* __restrict__ idx, int64_t cnt, const double* __restrict__ x,
                                        int64_t ldx, double* __restrict__ out, int nb) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int g = idx[t];
        for (int k = 0; k < nb; ++k) out[k * cnt + t] = x[k * ldx + g];
    }
}

void launch_gather_vec_multi(const int32_t* idx, int64_t cnt, const double* x, int64_t ldx, double* out, int nb,
                             cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t want = (cnt + 255) / 256;
    gather_vec_multi_kernel<<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(idx, cnt, x, ldx, out, nb);
}

void launch_gather_vec(const int32_t* idx, int64_t cnt, const double* x, double* out, cudaStream_t s) {
    if (cnt <= 0) return;
    const int64_t want = (cnt + 255) / 256;
    gather_vec_kernel<<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(idx, cnt, x, out);
}

// dst[dst_off[r] + c] = src[src_off[r] + c] for c < len[r]: copies rows of
// matrices with different leading dimensions.
template <typename T>
__global__ void gather_rows_kernel(const T* __restrict__ src, const int64_t* __restrict__ src_off,
                                   T* __restrict__ dst, const int64_t* __restrict__ dst_off,
                                   const int32_t* __restrict__ len, int64_t nrows) {
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const T* s = src + src_off[r];
        T* d = dst + dst_off[r];
        for (int c = threadIdx.x; c < len[r]; c += blockDim.x) d[c] = s[c];
    }
}

template <typename T>
void launch_gather_rows(const T* src, const int64_t* src_off, T* dst, const int64_t* dst_off, const int32_t* len,
                        int64_t nrows, cudaStream_t s) {
    if (nrows <= 0) return;
    gather_rows_kernel<T><<<(unsigned)(nrows < 65535 ? nrows : 65535), 128, 0, s>>>(src, src_off, dst, dst_off, len,
                                                                                     nrows);
}
template void launch_gather_rows<float>(const float*, const int64_t*, float*, const int64_t*, const int32_t*, int64_t,
                                        cudaStream_t);
template void launch_gather_rows<double>(const double*, const int64_t*, double*, const int64_t*, const int32_t*,
                                         int64_t, cudaStream_t);

// ------------------------------------------------------------------ prolongation
// z[g] = sum over the copies of g in the local vectors (fixed subdomain order)
//      + zc[t]   (the coarse prolongation (Z_i e_i)[a] of the owner i of g,
//                 a = position of g in Omega_Ii, t = off_I[i] + a: thread t
//                 runs in that owner order).  nb right-hand sides: yloc, zc
//                 and z hold nb vectors ldy, ldzc and ldz apart.
template <typename TY>
__global__ void __launch_bounds__(256) scatter_prolong_kernel(
    int64_t n, const int32_t* __restrict__ order_g, const int64_t* __restrict__ sc_ptr,
    const int32_t* __restrict__ sc_idx, const TY* __restrict__ yloc, const double* __restrict__ zc,
    double* __restrict__ z, int nb, int64_t ldy, int64_t ldzc, int64_t ldz) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int g = order_g[t];
        for (int r = 0; r < nb; ++r) {
            double s = 0.0;
            for (int64_t k = sc_ptr[g]; k < sc_ptr[g + 1]; ++k) s += (double)yloc[r * ldy + sc_idx[k]];
            if (zc) s += zc[r * ldzc + t];
            z[r * ldz + g] = s;
        }
    }
}

template <typename TY>
void launch_scatter_prolong(int64_t n, const int32_t* order_g, const int64_t* sc_ptr, const int32_t* sc_idx,
                            const TY* yloc, const double* zc, double* z, cudaStream_t s, int nb, int64_t ldy,
                            int64_t ldzc, int64_t ldz) {
    if (n <= 0) return;
    const int64_t want = (n + 255) / 256;
    scatter_prolong_kernel<TY><<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(
        n, order_g, sc_ptr, sc_idx, yloc, zc, z, nb, ldy, ldzc, ldz);
}
template void launch_scatter_prolong<float>(int64_t, const int32_t*, const int64_t*, const int32_t*, const float*,
                                            const double*, double*, cudaStream_t, int, int64_t, int64_t, int64_t);
template void launch_scatter_prolong<double>(int64_t, const int32_t*, const int64_t*, const int32_t*, const double*,
                                             const double*, double*, cudaStream_t, int, int64_t, int64_t, int64_t);

// ------------------------------------------------------------------ coarse blocks
// E[coff_i + r][coff_j + c] = sum_l Zt_i[r][la[l]] * AZ_j[lpos[l]][c], 32 x 32
// tile per CTA (i > j: strictly lower blocks of E).
__global__ void __launch_bounds__(256) e_offdiag_kernel(const EPairRef* __restrict__ tiles,
                                                         const int32_t* __restrict__ la,
                                                         const int32_t* __restrict__ lpos,
                                                         const double* __restrict__ Zt,
                                                         const int64_t* __restrict__ zt_off,
                                                         const int32_t* __restrict__ nI,
                                                         const double* __restrict__ AZ,
                                                         const int64_t* __restrict__ az_off,
                                                         const int32_t* __restrict__ p,
                                                         const int64_t* __restrict__ coff, double* __restrict__ E,
                                                         int64_t ldE) {
    const EPairRef t = tiles[blockIdx.x];
    const int pi = p[t.i], pj = p[t.j];
    const int ni = nI[t.i];
    const double* zt = Zt + zt_off[t.i];
    const double* az = AZ + az_off[t.j];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int c = t.tc * 32 + tx;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < t.list_len; ++l) {
        const int a = la[t.list_off + l], ps = lpos[t.list_off + l];
        const double bv = (c < pj) ? az[(size_t)ps * pj + c] : 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = t.tr * 32 + ty + 8 * q;
            if (r < pi) acc[q] = fma(zt[(size_t)r * ni + a], bv, acc[q]);
        }
    }
    if (c < pj) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = t.tr * 32 + ty + 8 * q;
            if (r < pi) E[(size_t)(coff[t.i] + r) * ldE + (coff[t.j] + c)] = acc[q];
        }
    }
}

void launch_e_offdiag(const EPairRef* tiles, int ntiles, const int32_t* la, const int32_t* lpos, const double* Zt,
                      const int64_t* zt_off, const int32_t* nI, const double* AZ, const int64_t* az_off,
                      const int32_t* p, const int64_t* coff, double* E, int64_t ldE, cudaStream_t s) {
    if (ntiles > 0)
        e_offdiag_kernel<<<ntiles, 256, 0, s>>>(tiles, la, lpos, Zt, zt_off, nI, AZ, az_off, p, coff, E, ldE);
}

// ------------------------------------------------------------------ reductions
// Fixed grid (DOT_BLOCKS x 256) and fixed per-thread strides, then a fixed
// tree in shared memory: the result is bitwise reproducible for a given n.
__device__ __forceinline__ double block_sum_256(double v) {
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

__global__ void __launch_bounds__(256) dot_partials_kernel(int64_t n, const double* __restrict__ x,
                                                            const double* __restrict__ y,
                                                            double* __restrict__ partials, int64_t ld) {
    x += (int64_t)blockIdx.y * ld;
    y += (int64_t)blockIdx.y * ld;
    partials += (int64_t)blockIdx.y * DOT_BLOCKS;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)DOT_BLOCKS * 256)
        s = fma(x[i], y[i], s);
    s = block_sum_256(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

void launch_dot_partials(int64_t n, const double* x, const double* y, double* partials, cudaStream_t s, int nb,
                         int64_t ld) {
    dot_partials_kernel<<<dim3(DOT_BLOCKS, nb), 256, 0, s>>>(n, x, y, partials, ld);
}

__global__ void __launch_bounds__(256) dot_finalize_kernel(const double* __restrict__ partials, PcgScal* sc,
                                                            int which, double tol2, int skip_done) {
    partials += (int64_t)blockIdx.x * DOT_BLOCKS;
    sc += blockIdx.x;
    if (skip_done && sc->conv) return;  // a converged right-hand side keeps its state
    double v = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += 256) v += partials[i];
    v = block_sum_256(v);
    if (threadIdx.x == 0) {
        switch (which) {
            case 0:
                sc->pq = v;
                sc->alpha = sc->rz / v;
                break;
            case 1:
                sc->rz_new = v;
                sc->beta = v / sc->rz;
                sc->rz = v;
                break;
            case 2:
                sc->rr = v;
                sc->iters += 1;
                sc->conv = (v <= tol2 * sc->bb) ? 1 : 0;
                break;
            case 3:
                sc->bb = v;
                break;
            case 4:
                sc->rz = v;
                break;
            default:
                sc->rr = v;
                sc->conv = (v <= tol2 * sc->bb) ? 1 : 0;
                break;
        }
    }
}

void launch_dot_finalize(const double* partials, PcgScal* sc, int which, double tol2, cudaStream_t s, int nb,
                         int skip_done) {
    dot_finalize_kernel<<<nb, 256, 0, s>>>(partials, sc, which, tol2, skip_done);
}

// x += alpha p; r -= alpha q; partial sums of r.r
__global__ void __launch_bounds__(256) pcg_update_xr_kernel(int64_t n, double* __restrict__ x,
                                                             double* __restrict__ r, const double* __restrict__ p,
                                                             const double* __restrict__ q,
                                                             const PcgScal* __restrict__ sc,
                                                             double* __restrict__ partials, int64_t ld,
                                                             int skip_done) {
    const int k = blockIdx.y;
    if (skip_done && sc[k].conv) return;
    x += (int64_t)k * ld;
    r += (int64_t)k * ld;
    p += (int64_t)k * ld;
    q += (int64_t)k * ld;
    partials += (int64_t)k * DOT_BLOCKS;
    const double a = sc[k].alpha;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)DOT_BLOCKS * 256) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        s = fma(ri, ri, s);
    }
    s = block_sum_256(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

void launch_pcg_update_xr(int64_t n, double* x, double* r, const double* p, const double* q, const PcgScal* sc,
                          double* partials, cudaStream_t s, int nb, int64_t ld, int skip_done) {
    pcg_update_xr_kernel<<<dim3(DOT_BLOCKS, nb), 256, 0, s>>>(n, x, r, p, q, sc, partials, ld, skip_done);
}

// p = z + beta p
__global__ void pcg_update_p_kernel(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                                    const PcgScal* __restrict__ sc, int64_t ld, int skip_done) {
    const int k = blockIdx.y;
    if (skip_done && sc[k].conv) return;
    p += (int64_t)k * ld;
    z += (int64_t)k * ld;
    const double b = sc[k].beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(b, p[i], z[i]);
}

void launch_pcg_update_p(int64_t n, double* p, const double* z, const PcgScal* sc, cudaStream_t s, int nb,
                         int64_t ld, int skip_done) {
    pcg_update_p_kernel<<<dim3(DOT_BLOCKS, nb), 256, 0, s>>>(n, p, z, sc, ld, skip_done);
}

// End of one PCG iteration replayed inside a CUDA graph's while-loop: log the
// step length alpha of the iteration just finished (and the ratio beta that
// built its direction, from the second iteration on) for the Lanczos
// condition estimate, and continue the loop while the recursive residual is
// above the tolerance and fewer than *maxit iterations have run.
__global__ void pcg_loop_cond_kernel(const PcgScal* __restrict__ sc, const int* __restrict__ maxit,
                                     double* __restrict__ alog, double* __restrict__ blog,
                                     cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0) return;
    const int k = sc->iters;
    if (k >= 1 && k <= *maxit) alog[k - 1] = sc->alpha;
    if (k >= 2 && k <= *maxit) blog[k - 2] = sc->beta;
    cudaGraphSetConditional(loop, (!sc->conv && k < *maxit) ? 1u : 0u);
}

void launch_pcg_loop_cond(const PcgScal* sc, const int* maxit, double* alog, double* blog,
                          cudaGraphConditionalHandle loop, cudaStream_t s) {
    pcg_loop_cond_kernel<<<1, 32, 0, s>>>(sc, maxit, alog, blog, loop);
}

// out = a x + b y
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fma(a, x[i], b * y[i]);
}

void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
    if (n > 0) axpby_kernel<<<DOT_BLOCKS, 256, 0, s>>>(n, a, x, b, y, out);
}

}  // namespace amdd
