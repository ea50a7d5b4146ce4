// Kernels of the learned warm start of the local eigensolve (the eigenvectors
// of eq. (Zi) when the selection is partial) and of the block LOBPCG that
// uses it:
//   * subdomain features (32 statistics of A_ii and the sizes) and the
//     orthonormal Krylov basis K_16(A_II, 1) on which proposals are expressed;
//   * the MLP (32 -> 256 -> 256 -> 256, ReLU; weights held at bfloat16
//     precision, FP32 arithmetic): bias / activation, symmetrisation of the
//     output as a 16 x 16 matrix, the squared-error loss and its gradient,
//     ReLU backward, bias gradients (fixed-order sums) and the Adam update
//     followed by rounding of the weights to bfloat16;
//   * row helpers of LOBPCG: counter-based random rows, residual rows with
//     their norms, unit-normalised rows, rows scaled by w^{-1/2}.
// The dense products of both the MLP and LOBPCG run on the batched GEMM.
#include "amdd_internal.h"

namespace amdd {

// ------------------------------------------------------------------ features
namespace {

struct Acc4 {  // sum, sum of squares, min, max
    double s, q, mn, mx;
    __device__ void init() {
        s = 0.0;
        q = 0.0;
        mn = 1e300;
        mx = -1e300;
    }
    __device__ void add(double v) {
        s += v;
        q += v * v;
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
};

__device__ double block_sum_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}
__device__ double block_min_d(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmin(t, sh[w]);
    return t;
}
__device__ double block_max_d(double v, double* sh) { return -block_min_d(-v, sh); }

}  // namespace

// One CTA per subdomain.  The definitions follow the statistics listed in
// amdd_internal.h (FeatDesc); every one is a symmetric function of the
// unknowns of Omega_I.
__global__ void __launch_bounds__(256) features_kernel(const FeatDesc* __restrict__ descs) {
    const FeatDesc d = descs[blockIdx.x];
    __shared__ double sh[8];
    const int nI = d.nI, ld = d.ld, nc = d.ncols;
    Acc4 ldg, lof, dom;
    ldg.init();
    lof.init();
    dom.init();
    double deg_s = 0.0, deg_q = 0.0, deg_mx = 0.0, cg_pos = 0.0, cg_s = 0.0, cg_mx = 0.0, fro = 0.0, tr = 0.0;
    double npos = 0.0, nnz = 0.0, bnd_n = 0.0, bnd_ld = 0.0;
    for (int r = threadIdx.x; r < nI; r += blockDim.x) {
        const double* row = d.A + (size_t)r * ld;
        const double dr = row[r];
        double offabs = 0.0, cg = 0.0, deg = 0.0;
        for (int c = 0; c < nI; ++c) {
            const double v = row[c];
            fro += v * v;
            if (c == r || v == 0.0) continue;
            offabs += fabs(v);
            deg += 1.0;
            nnz += 1.0;
            if (v > 0.0) npos += 1.0;
            lof.add(log(fabs(v)));
        }
        for (int c = nI; c < nc; ++c) cg += fabs(row[c]);
        cg /= dr;
        const double l = log(dr);
        ldg.add(l);
        dom.add(offabs / dr);
        deg_s += deg;
        deg_q += deg * deg;
        deg_mx = fmax(deg_mx, deg);
        if (cg > 0.0) {
            cg_pos += 1.0;
            bnd_n += 1.0;
            bnd_ld += l;
        }
        cg_s += cg;
        cg_mx = fmax(cg_mx, cg);
        tr += dr;
    }
    const double n = (double)nI;
    double f[32];
    f[0] = log(n);
    f[1] = log1p((double)d.nG);
    f[2] = log1p((double)d.nD);
    f[3] = d.nG / n;
    f[4] = d.nD / n;
    auto stats = [&](Acc4& a, double cnt, int at) {
        const double s = block_sum_d(a.s, sh), q = block_sum_d(a.q, sh);
        const double mn = block_min_d(a.mn, sh), mx = block_max_d(a.mx, sh);
        if (cnt > 0.0) {
            const double m = s / cnt;
            f[at] = m;
            f[at + 1] = sqrt(fmax(q / cnt - m * m, 0.0));
            f[at + 2] = mn;
            f[at + 3] = mx;
        } else {
            f[at] = f[at + 1] = f[at + 2] = f[at + 3] = 0.0;
        }
    };
    const double nnz_t = block_sum_d(nnz, sh);
    stats(ldg, n, 5);
    stats(lof, nnz_t, 9);
    f[13] = f[8] - f[7];
    const double ds = block_sum_d(deg_s, sh), dq = block_sum_d(deg_q, sh);
    f[14] = ds / n;
    f[15] = sqrt(fmax(dq / n - f[14] * f[14], 0.0));
    f[16] = block_max_d(deg_mx, sh);
    f[17] = block_sum_d(cg_pos, sh) / n;
    f[18] = block_sum_d(cg_s, sh) / n;
    f[19] = block_max_d(cg_mx, sh);
    stats(dom, n, 20);
    f[24] = log(sqrt(block_sum_d(fro, sh)) / n);
    f[25] = log(block_sum_d(tr, sh) / n);
    const double np_ = block_sum_d(npos, sh);
    f[26] = nnz_t > 0.0 ? np_ / nnz_t : 0.0;
    f[27] = log(fmax((double)d.p, 1.0) / n);
    f[28] = log(fmax((double)d.p, 1.0));
    f[29] = log(d.tau);
    const double bn = block_sum_d(bnd_n, sh), bl = block_sum_d(bnd_ld, sh);
    f[30] = bn > 0.0 ? bl / bn - f[5] : 0.0;
    f[31] = 1.0;
    if (threadIdx.x < 32) d.out[threadIdx.x] = (float)f[threadIdx.x];
}

void launch_features(const FeatDesc* d, int nmat, cudaStream_t s) {
    if (nmat > 0) features_kernel<<<nmat, 256, 0, s>>>(d);
}

// Orthonormal basis of K_16(A_II, 1), one CTA per subdomain, as rows of Bt
// (16 x nI): v_0 = 1/sqrt(nI); v_j = A_II v_{j-1}, classical Gram-Schmidt
// against v_0..v_{j-1} applied twice, normalised; a vector whose norm drops
// below 1e-12 of its norm before orthogonalisation ends the space (the rest
// of the rows are zero).  w is a scratch row of nI entries.
__global__ void __launch_bounds__(256) krylov_kernel(const KrylovDesc* __restrict__ descs) {
    const KrylovDesc d = descs[blockIdx.x];
    __shared__ double sh[8];
    __shared__ double hco[PROP_NB];
    const int nI = d.nI;
    const double v0 = rsqrt((double)nI);
    for (int r = threadIdx.x; r < nI; r += blockDim.x) d.Bt[r] = v0;
    for (int j = 1; j < PROP_NB; ++j)
        for (int r = threadIdx.x; r < nI; r += blockDim.x) d.Bt[(size_t)j * nI + r] = 0.0;
    __syncthreads();
    bool done = false;
    for (int j = 1; j < PROP_NB && !done; ++j) {
        const double* prev = d.Bt + (size_t)(j - 1) * nI;
        double part = 0.0;
        for (int r = threadIdx.x; r < nI; r += blockDim.x) {
            const double* row = d.A + (size_t)r * d.ld;
            double s = 0.0;
            for (int c = 0; c < nI; ++c) s = fma(row[c], prev[c], s);
            d.w[r] = s;
            part += s * s;
        }
        __syncthreads();
        const double w0 = sqrt(block_sum_d(part, sh));
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < j; ++l) {
                const double* bl = d.Bt + (size_t)l * nI;
                double s = 0.0;
                for (int r = threadIdx.x; r < nI; r += blockDim.x) s = fma(bl[r], d.w[r], s);
                s = block_sum_d(s, sh);
                if (threadIdx.x == 0) hco[l] = s;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < nI; r += blockDim.x) {
                double s = d.w[r];
                for (int l = 0; l < j; ++l) s = fma(-hco[l], d.Bt[(size_t)l * nI + r], s);
                d.w[r] = s;
            }
            __syncthreads();
        }
        double part2 = 0.0;
        for (int r = threadIdx.x; r < nI; r += blockDim.x) part2 += d.w[r] * d.w[r];
        const double nw = sqrt(block_sum_d(part2, sh));
        if (!(nw > 1e-12 * w0)) {
            done = true;
        } else {
            const double inv = 1.0 / nw;
            for (int r = threadIdx.x; r < nI; r += blockDim.x) d.Bt[(size_t)j * nI + r] = d.w[r] * inv;
        }
        __syncthreads();
    }
}

void launch_krylov(const KrylovDesc* d, int nmat, cudaStream_t s) {
    if (nmat > 0) krylov_kernel<<<nmat, 256, 0, s>>>(d);
}

// ------------------------------------------------------------------ MLP
// bfloat16 rounding of binary32: add 0x7FFF plus the lowest kept bit, keep
// the top 16 bits (nearest, ties to even); NaN stays NaN.
__device__ __forceinline__ float bf16_round(float x) {
    if (x != x) return x;
    unsigned u = __float_as_uint(x);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(u);
}

// X[b][f] = (feat[b][f] - mean[f]) / sd[f]
__global__ void normalize_features_kernel(const float* __restrict__ feat, const float* __restrict__ mean,
                                          const float* __restrict__ sd, float* __restrict__ X, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * PROP_NF; t += gridDim.x * blockDim.x) {
        const int f = t % PROP_NF;
        X[t] = (feat[t] - mean[f]) / sd[f];
    }
}

// Standardisation of the features: per column f of the n x PROP_NF matrix,
// mean and population standard deviation (two passes, FP64 sums in a fixed
// order: one thread per column strides the rows, then a fixed tree over the
// 8 threads of the column); sd below 1e-6 becomes 1 so that a constant
// feature passes unchanged.
__global__ void __launch_bounds__(256) feature_stats_kernel(const float* __restrict__ feat, int n,
                                                            float* __restrict__ mean, float* __restrict__ sd) {
    __shared__ double red[8][PROP_NF];
    __shared__ double mu_s[PROP_NF];
    const int f = threadIdx.x % PROP_NF, part = threadIdx.x / PROP_NF;  // 8 parts x 32 columns
    double s = 0.0;
    for (int r = part; r < n; r += 8) s += feat[(size_t)r * PROP_NF + f];
    red[part][f] = s;
    __syncthreads();
    if (part == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q][f];
        mu_s[f] = t / n;
    }
    __syncthreads();
    const double mu = mu_s[f];
    double v = 0.0;
    for (int r = part; r < n; r += 8) {
        const double d = feat[(size_t)r * PROP_NF + f] - mu;
        v += d * d;
    }
    __syncthreads();
    red[part][f] = v;
    __syncthreads();
    if (part == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q][f];
        const double sdv = sqrt(t / n);
        mean[f] = (float)mu;
        sd[f] = sdv > 1e-6 ? (float)sdv : 1.0f;
    }
}

void launch_feature_stats(const float* feat, int n, float* mean, float* sd, cudaStream_t s) {
    feature_stats_kernel<<<1, 8 * PROP_NF, 0, s>>>(feat, n, mean, sd);
}

void launch_normalize_features(const float* feat, const float* mean, const float* sd, float* X, int n,
                               cudaStream_t s) {
    if (n > 0) normalize_features_kernel<<<(n * PROP_NF + 255) / 256, 256, 0, s>>>(feat, mean, sd, X, n);
}

// Z[b][j] += bias[j]; H = relu(Z) when H is given (Z keeps the pre-activation)
__global__ void bias_act_kernel(float* __restrict__ Z, const float* __restrict__ bias, float* __restrict__ H, int rows,
                                int cols) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows * cols; t += gridDim.x * blockDim.x) {
        const float z = Z[t] + bias[t % cols];
        Z[t] = z;
        if (H) H[t] = fmaxf(z, 0.0f);
    }
}

void launch_bias_act(float* Z, const float* bias, float* H, int rows, int cols, cudaStream_t s) {
    const int n = rows * cols;
    if (n > 0) bias_act_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(Z, bias, H, rows, cols);
}

// Q[b] = (Y[b] + Y[b]^T) / 2 as 16 x 16 matrices
__global__ void symmetrise_kernel(const float* __restrict__ Y, float* __restrict__ Q, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * PROP_NO; t += gridDim.x * blockDim.x) {
        const int b = t / PROP_NO, e = t % PROP_NO, r = e / PROP_NB, c = e % PROP_NB;
        const float* y = Y + (size_t)b * PROP_NO;
        Q[t] = 0.5f * (y[r * PROP_NB + c] + y[c * PROP_NB + r]);
    }
}

void launch_symmetrise(const float* Y, float* Q, int n, cudaStream_t s) {
    if (n > 0) symmetrise_kernel<<<(n * PROP_NO + 255) / 256, 256, 0, s>>>(Y, Q, n);
}

// Loss sum_b ||Q_b - Qt_b||_F^2 / n (partial sums per CTA, row b) and the
// gradient with respect to the unsymmetrised outputs:
// dY = (dQ + dQ^T) / 2 with dQ = 2 (Q - Qt) / n.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ Q, const float* __restrict__ Qt,
                                                        float* __restrict__ dY, float* __restrict__ part, int n) {
    __shared__ float sh[8];
    const int b = blockIdx.x;
    const float* q = Q + (size_t)b * PROP_NO;
    const float* qt = Qt + (size_t)b * PROP_NO;
    float acc = 0.0f;
    for (int e = threadIdx.x; e < PROP_NO; e += blockDim.x) {
        const int r = e / PROP_NB, c = e % PROP_NB;
        const float dqe = q[e] - qt[e];
        const float dqt = q[c * PROP_NB + r] - qt[c * PROP_NB + r];
        acc = fmaf(dqe, dqe, acc);
        dY[(size_t)b * PROP_NO + e] = (dqe + dqt) / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[b] = t;
    }
}

// loss = sum of the per-sample partials / n, in sample order
__global__ void loss_finalize_kernel(const float* __restrict__ part, float* __restrict__ out, int n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < n; ++b) t += part[b];
        out[0] = (float)(t / n);
    }
}

void launch_loss_grad(const float* Q, const float* Qt, float* dY, float* part, float* loss, int n, cudaStream_t s) {
    if (n <= 0) return;
    loss_grad_kernel<<<n, 256, 0, s>>>(Q, Qt, dY, part, n);
    loss_finalize_kernel<<<1, 32, 0, s>>>(part, loss, n);
}

// dZ = dH * (Z > 0)
__global__ void relu_back_kernel(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                                 int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        dZ[t] = Z[t] > 0.0f ? dH[t] : 0.0f;
}

void launch_relu_back(const float* dH, const float* Z, float* dZ, int n, cudaStream_t s) {
    if (n > 0) relu_back_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(dH, Z, dZ, n);
}

// db[j] = sum_b dZ[b][j], summed in sample order
__global__ void colsum_kernel(const float* __restrict__ dZ, float* __restrict__ db, int rows, int cols) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.0f;
    for (int b = 0; b < rows; ++b) s += dZ[(size_t)b * cols + j];
    db[j] = s;
}

void launch_colsum(const float* dZ, float* db, int rows, int cols, cudaStream_t s) {
    if (cols > 0) colsum_kernel<<<(cols + 127) / 128, 128, 0, s>>>(dZ, db, rows, cols);
}

// Adam (Kingma & Ba) on the FP32 master weights, then the bfloat16-rounded copy
__global__ void adam_kernel(float* __restrict__ W, float* __restrict__ Wb, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.0f - b1) * gt;
        const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        const float w = W[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
        W[t] = w;
        Wb[t] = bf16_round(w);
    }
}

void launch_adam(float* W, float* Wb, float* m, float* v, const float* g, int n, float lr, int t, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(W, Wb, m, v, g, n, lr, b1, b2, 1e-8f,
                                                                                c1, c2);
}

__global__ void bf16_round_kernel(const float* __restrict__ W, float* __restrict__ Wb, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) Wb[t] = bf16_round(W[t]);
}

void launch_bf16_round(const float* W, float* Wb, int n, cudaStream_t s) {
    if (n > 0) bf16_round_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(W, Wb, n);
}

// ------------------------------------------------------------------ LOBPCG rows
// splitmix64 (Steele, Lea & Flood, 2014) of a counter: uniform in [-1, 1)
__device__ __forceinline__ double counter_uniform(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// rows [r0, r1) of each matrix filled from the counter (seed, matrix id, row, column)
template <typename T>
__global__ void rng_rows_kernel(const RowsDesc<T>* __restrict__ descs, unsigned long long seed) {
    const RowsDesc<T> d = descs[blockIdx.y];
    for (int r = d.r0 + blockIdx.x; r < d.r1; r += gridDim.x)
        for (int c = threadIdx.x; c < d.cols; c += blockDim.x) {
            const unsigned long long ctr =
                seed ^ ((unsigned long long)d.id << 40) ^ ((unsigned long long)r << 20) ^ (unsigned long long)c;
            d.A[(size_t)r * d.ld + c] = (T)counter_uniform(ctr);
        }
}

template <typename T>
void launch_rng_rows(const RowsDesc<T>* d, int nmat, int maxrows, unsigned long long seed, cudaStream_t s) {
    if (nmat <= 0 || maxrows <= 0) return;
    dim3 grid(maxrows < 1024 ? maxrows : 1024, nmat);
    rng_rows_kernel<T><<<grid, 128, 0, s>>>(d, seed);
}
template void launch_rng_rows<float>(const RowsDesc<float>*, int, int, unsigned long long, cudaStream_t);
template void launch_rng_rows<double>(const RowsDesc<double>*, int, int, unsigned long long, cudaStream_t);

// R = TX - diag(theta) X (rows); norms of the first `want` residual rows
template <typename T>
__global__ void __launch_bounds__(256) residual_rows_kernel(const ResidDesc<T>* __restrict__ descs) {
    const ResidDesc<T> d = descs[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < d.k; r += 8) {
        const T th = d.theta[r];
        const T* x = d.X + (size_t)r * d.ld;
        const T* tx = d.TX + (size_t)r * d.ld;
        T* rr = d.R + (size_t)r * d.ld;
        T s = T(0);
        for (int c = lane; c < d.n; c += 32) {
            const T v = fma(-th, x[c], tx[c]);
            rr[c] = v;
            s = fma(v, v, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && r < d.want) d.norms[r] = (double)sqrt(s);
    }
}

template <typename T>
void launch_residual_rows(const ResidDesc<T>* d, int nmat, cudaStream_t s) {
    if (nmat > 0) residual_rows_kernel<T><<<nmat, 256, 0, s>>>(d);
}
template void launch_residual_rows<float>(const ResidDesc<float>*, int, cudaStream_t);
template void launch_residual_rows<double>(const ResidDesc<double>*, int, cudaStream_t);

// rows scaled: A[r] *= f[r] (f[r] = 0 zeroes the row); with unit != 0, f is
// 1 / ||A[r]|| (rows of zero norm stay zero)
template <typename T>
__global__ void __launch_bounds__(256) scale_rows_kernel(const ScaleDesc<T>* __restrict__ descs, int unit) {
    const ScaleDesc<T> d = descs[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < d.rows; r += 8) {
        T* a = d.A + (size_t)r * d.ld;
        T f;
        if (unit) {
            T s = T(0);
            for (int c = lane; c < d.cols; c += 32) s = fma(a[c], a[c], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            f = s > T(0) ? T(1) / sqrt(s) : T(0);
        } else {
            f = d.f[r];
        }
        for (int c = lane; c < d.cols; c += 32) a[c] *= f;
    }
}

template <typename T>
void launch_scale_rows(const ScaleDesc<T>* d, int nmat, int unit, cudaStream_t s) {
    if (nmat > 0) scale_rows_kernel<T><<<nmat, 256, 0, s>>>(d, unit);
}
template void launch_scale_rows<float>(const ScaleDesc<float>*, int, int, cudaStream_t);
template void launch_scale_rows<double>(const ScaleDesc<double>*, int, int, cudaStream_t);

// entries above the diagonal of rows [r0, r1) set to zero (a lower factor
// stored in a matrix whose upper triangle still holds the input)
// out[t] = sum_c W[off[t] + c] W[off[t] + len[t] + c]: the dot product of the
// two halves of a row, one warp per row
template <typename T>
__global__ void __launch_bounds__(256) half_dots_kernel(const T* __restrict__ W, const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ len, int64_t rows,
                                                        double* __restrict__ out) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= rows) return;  // whole warps
    const T* a = W + off[t];
    const int L = len[t];
    double s = 0.0;
    for (int c = lane; c < L; c += 32) s = fma((double)a[c], (double)a[L + c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[t] = s;
}

template <typename T>
void launch_half_dots(const T* W, const int64_t* off, const int32_t* len, int64_t rows, double* out, cudaStream_t s) {
    if (rows > 0) half_dots_kernel<T><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(W, off, len, rows, out);
}
template void launch_half_dots<float>(const float*, const int64_t*, const int32_t*, int64_t, double*, cudaStream_t);
template void launch_half_dots<double>(const double*, const int64_t*, const int32_t*, int64_t, double*, cudaStream_t);

template <typename T>
__global__ void zero_upper_kernel(const RowsDesc<T>* __restrict__ descs) {
    const RowsDesc<T> d = descs[blockIdx.y];
    for (int r = d.r0 + blockIdx.x; r < d.r1; r += gridDim.x)
        for (int c = r + 1 + threadIdx.x; c < d.cols; c += blockDim.x) d.A[(size_t)r * d.ld + c] = T(0);
}

template <typename T>
void launch_zero_upper(const RowsDesc<T>* d, int nmat, int maxrows, cudaStream_t s) {
    if (nmat <= 0 || maxrows <= 0) return;
    dim3 grid(maxrows < 1024 ? maxrows : 1024, nmat);
    zero_upper_kernel<T><<<grid, 128, 0, s>>>(d);
}
template void launch_zero_upper<float>(const RowsDesc<float>*, int, int, cudaStream_t);
template void launch_zero_upper<double>(const RowsDesc<double>*, int, int, cudaStream_t);

}  // namespace amdd
