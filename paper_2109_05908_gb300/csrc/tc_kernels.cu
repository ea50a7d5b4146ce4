// Batched FP32 GEMM on the fifth-generation tensor cores (tcgen05, sm_103a):
// C = alpha op(A) op(B) + beta C for every descriptor of a batch, one CTA per
// 128 x 128 output tile.
//
// FP32 accuracy from TF32 units ("3xTF32"): each operand value v is split as
// v = hi + lo with hi = tf32(v) (round to nearest) and lo = tf32(v - hi), and
// the product is accumulated as hi_a hi_b + hi_a lo_b + lo_a hi_b; the
// dropped lo_a lo_b term is below 2^-21 of |a b|.  The tensor core's own
// accumulation over long k is less accurate than IEEE FP32 (measured: 5 to
// 10 times the error of an FP32 multiply-add loop at k = 1000 to 2048), so
// the tensor memory holds the product of one 32-wide k chunk at a time, and
// the chunks are summed in FP32 registers, one output row per thread.
//
// Per chunk the 128 threads load op(A) and op(B) (coalesced for either
// storage order), split them, and store hi and lo into shared memory in the
// 128-byte-swizzled K-major layout of the tensor core's shared-memory
// descriptors (8-row atoms of 1024 bytes; the 16-byte chunk c of row r sits at
// chunk position c ^ (r mod 8)).  One elected thread issues the 4 x 3
// tcgen05.mma (M = 128, N = 128, K = 8 each) into one of two tensor-memory
// buffers and commits them to an mbarrier that every thread waits on, with an
// iteration limit, before the tiles are rewritten; while the chunk runs the
// threads add the previous chunk's buffer (tcgen05.ld: warp w owns lanes
// 32 w .. 32 w + 31, i.e. output rows) into their registers.  The epilogue
// applies alpha, beta and the lower-triangle mask.
#include "amdd_internal.h"
#include "jacobi_pair_inner.cuh"

namespace amdd {

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 128;
constexpr int TC_KC = 32;                       // k per chunk: one 128-byte swizzle row of FP32
constexpr int TC_TILE_BYTES = TC_M * TC_KC * 4; // 16 KB per operand tile
constexpr unsigned TC_WAIT_LIMIT = 1u << 24;    // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, k) in a 128B-swizzled K-major tile of FP32 with 32 k per row
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + (((k >> 2) ^ (r & 7)) << 4) + (k & 3) * 4);
}

// shared-memory matrix descriptor: start address, leading byte offset (unused
// for swizzled K-major), stride byte offset between 8-row atoms, descriptor
// version 1, layout type 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (unsigned it = 0; it < TC_WAIT_LIMIT && !done; ++it)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
    return done != 0;
}

// Block flags of the persistent block-pair sweep: bounded acquire wait until
// *f >= v (about a second of polling), and a release store.
__device__ __forceinline__ bool flag_wait_geq(const int* f, int v, long long limit = 2000000000ll) {
    const long long start = clock64();
    for (;;) {
        int x;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(x) : "l"(f) : "memory");
        if (x >= v) return true;
        if (clock64() - start > limit) return false;
        __nanosleep(64);
    }
}
__device__ __forceinline__ void flag_publish(int* f, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

}  // namespace

// acc[j] += the 32-bit values of columns c0 .. c0 + 15 of this warp's lanes of
// tensor memory at taddr
__device__ __forceinline__ void tmem_add16(uint32_t taddr, float* acc) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(v[j]);
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmDescT<float>* __restrict__ descs,
                                                      const TileRef* __restrict__ tiles, int ntiles,
                                                      int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* base = tc_raw + ((1024 - (smem_u32(tc_raw) & 1023)) & 1023);
    unsigned char* Ahi = base;
    unsigned char* Alo = base + TC_TILE_BYTES;
    unsigned char* Bhi = base + 2 * TC_TILE_BYTES;
    unsigned char* Blo = base + 3 * TC_TILE_BYTES;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const TileRef tr = tiles[t];
    const GemmDescT<float> d = descs[tr.desc];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row0 = tr.tm * TC_M, col0 = tr.tn * TC_N;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    // D f32, A and B tf32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    const uint32_t mb = smem_u32(&mbar);

    float acc[TC_N];
#pragma unroll
    for (int j = 0; j < TC_N; ++j) acc[j] = 0.0f;
    int kbeg = 0;
    if (d.kfrom_row) kbeg = (row0 / TC_KC) * TC_KC;
    uint32_t chunk = 0;
    for (int k0 = kbeg; k0 < d.k; k0 += TC_KC, ++chunk) {
        if (chunk > 0) {
            // the previous chunk's MMAs are done before its tiles are rewritten
            const bool mine = mbar_wait(mb, (chunk - 1) & 1u);
            if (!__syncthreads_and(mine ? 1 : 0)) {
                if (tid == 0) failed = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        // op(A)[row0 + r][k0 + kk] and op(B)^T[col0 + c][k0 + kk]
        for (int e = tid; e < TC_M * TC_KC; e += 128) {
            int r, kk;
            if (!d.ta) {
                r = e / TC_KC;
                kk = e % TC_KC;
            } else {
                kk = e / TC_M;
                r = e % TC_M;
            }
            const int gr = row0 + r, gk = k0 + kk;
            float v = 0.0f;
            if (gr < d.m && gk < d.k) v = d.ta ? d.A[(size_t)gk * d.lda + gr] : d.A[(size_t)gr * d.lda + gk];
            const float hi = tf32_rna(v);
            const uint32_t o = sw128_off(r, kk);
            *reinterpret_cast<float*>(Ahi + o) = hi;
            *reinterpret_cast<float*>(Alo + o) = tf32_rna(v - hi);
        }
        for (int e = tid; e < TC_N * TC_KC; e += 128) {
            int c, kk;
            if (d.tb) {
                c = e / TC_KC;
                kk = e % TC_KC;
            } else {
                kk = e / TC_N;
                c = e % TC_N;
            }
            const int gc = col0 + c, gk = k0 + kk;
            float v = 0.0f;
            if (gc < d.n && gk < d.k) v = d.tb ? d.B[(size_t)gc * d.ldb + gk] : d.B[(size_t)gk * d.ldb + gc];
            const float hi = tf32_rna(v);
            const uint32_t o = sw128_off(c, kk);
            *reinterpret_cast<float*>(Bhi + o) = hi;
            *reinterpret_cast<float*>(Blo + o) = tf32_rna(v - hi);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dbuf = tmem + (chunk & 1u) * TC_N;
        if (tid == 0) {
            for (int ks = 0; ks < TC_KC / 8; ++ks) {
                const uint32_t koff = (uint32_t)ks * 32;
                const uint64_t ah = sw128_desc(smem_u32(Ahi) + koff), al = sw128_desc(smem_u32(Alo) + koff);
                const uint64_t bh = sw128_desc(smem_u32(Bhi) + koff), bl = sw128_desc(smem_u32(Blo) + koff);
                mma_tf32(dbuf, ah, bh, idesc, ks > 0 ? 1u : 0u);
                mma_tf32(dbuf, ah, bl, idesc, 1u);
                mma_tf32(dbuf, al, bh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
        }
        if (chunk > 0) {
            // sum the previous chunk's product (done: waited above) while this one runs
            const uint32_t prev = tmem + ((chunk - 1) & 1u) * TC_N + lane_off;
#pragma unroll
            for (int q = 0; q < TC_N / 16; ++q) tmem_add16(prev + 16 * q, acc + 16 * q);
        }
    }
    if (!failed && chunk > 0) {
        const bool mine = mbar_wait(mb, (chunk - 1) & 1u);
        if (!__syncthreads_and(mine ? 1 : 0)) {
            if (tid == 0) failed = 1;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t last = tmem + ((chunk - 1) & 1u) * TC_N + lane_off;
#pragma unroll
            for (int q = 0; q < TC_N / 16; ++q) tmem_add16(last + 16 * q, acc + 16 * q);
        }
    }
    __syncthreads();
    if (failed) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
    } else {
        // epilogue (k = 0 leaves acc = 0: C = beta C)
        const int r = row0 + 32 * warp + lane;
        if (r < d.m) {
#pragma unroll
            for (int j = 0; j < TC_N; ++j) {
                const int c = col0 + j;
                if (c >= d.n || (d.lower && c > r)) continue;
                float* cp = d.C + (size_t)r * d.ldc + c;
                const float val = d.alpha * acc[j];
                *cp = (d.beta != 0.0f) ? fmaf(d.beta, *cp, val) : val;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
}

// ------------------------------------------------------------------ block-pair Jacobi on tensor cores
// One round of the block-pair one-sided Jacobi (the FP32 form of
// jacobi_pair_kernel, the same schedule, tests and inner eigensolve) with its
// two contractions on the tensor cores, in the same split as the GEMM above:
//   * Gram matrix of the pair's 64 rows Y over ncols_dot columns, in chunks of
//     64: the tile [hi(Y); lo(Y)] (128 rows, K-major, 128-byte swizzle, two
//     32-wide k atoms) times hi(Y)^T gives [hi hi^T; lo hi^T] by M = 128,
//     N = 64 MMAs, so G = hh + lh + lh^T (the dropped lo lo^T is below 2^-21
//     of |Y_p||Y_q|); each chunk's product is summed into FP32 registers while
//     the next chunk runs (two tensor-memory buffers, two staging tiles);
//   * rotation Y <- Qt Y over ncols_rot columns in chunks of 128, computed
//     transposed: D = Y_c^T Qt^T (M = 128 columns of Y, N = 64, K = 64) with
//     the 3 terms hi hi, hi lo, lo hi.  Y_c^T is staged K-major (the rows of Y
//     become the k index); in tensor memory lane c then holds column c of the
//     new rows, so every thread stores its column's entries and each warp
//     store covers 32 consecutive columns of one row.
// Every wait on the tensor core is bounded; on a timeout the CTA latches
// DERR_TIMEOUT, waits once more for its last commit and frees its tensor
// memory.  Shared memory: region X (the two Gram staging tiles, then the
// Gram buffers and Qt of the eigensolve, then hi/lo of Y_c^T) and region Q
// (hi/lo of Qt, the B operand of the rotation).
namespace {
constexpr int JT_KC = 64;                   // Gram: columns per chunk (two k atoms)
constexpr int JT_NC = 128;                  // rotation: columns per chunk (M of the MMA)
constexpr int JT_X = 64 * 1024;             // region X
constexpr int JT_Q = 32 * 1024;             // region Q
constexpr int JT_QT_OFF = 33 * 1024;        // Qt (FP32) inside region X, after G0 and G1
constexpr int JT_TMEM_COLS = 128;
static_assert(2 * JPI_N * JPI_LDG * 4 <= JT_QT_OFF, "Gram buffers before Qt");
static_assert(JT_QT_OFF + JPI_N * JPI_LDQ * 4 <= JT_X, "Qt in region X");
}  // namespace

__global__ void __maxnreg__(120) jacobi_pair_tc_kernel(const JacobiDescT<float>* __restrict__ descs,
                                                                const int4* __restrict__ tasks, int ntasks,
                                                                int* __restrict__ counter, int* __restrict__ bdone,
                                                                const int* __restrict__ bofs, float tol,
                                                                int inner_max, int* __restrict__ rotated,
                                                                unsigned long long* __restrict__ rots,
                                                                unsigned long long* __restrict__ stats,
                                                                int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char jt_raw[];
    unsigned char* base = jt_raw + ((1024 - (smem_u32(jt_raw) & 1023)) & 1023);
    unsigned char* rx = base;         // region X
    unsigned char* rq = base + JT_X;  // region Q
    float* G0 = reinterpret_cast<float*>(rx);
    float* G1 = G0 + JPI_N * JPI_LDG;
    float* Qt = reinterpret_cast<float*>(rx + JT_QT_OFF);
    __shared__ JpRound<float> jr[2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    __shared__ int task_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(JT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t mb = smem_u32(&mbar);
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t ncommit = 0;  // commits issued (the same count in every thread)
    bool ok = true;        // no wait timed out (uniform)
    const long long tlife = clock64();
    int ntask = 0;

    for (;;) {
        // ---- claim the next task (tasks are ordered by round) and wait until the
        // two row blocks have finished the previous round
        if (tid == 0) task_s = atomicAdd(counter, 1);
        __syncthreads();
        const int task = task_s;
        if (task >= ntasks) break;
        const int4 tk = tasks[task];
        const int mat = tk.x, kp = tk.y, nblk = tk.z, round = tk.w;
        const JacobiDescT<float> d = descs[mat];
        int bp, bq;
        if (kp == 0) {
            bp = nblk - 1;
            bq = round;
        } else {
            bp = (round + kp) % (nblk - 1);
            bq = (round - kp + nblk - 1) % (nblk - 1);
        }
        int* const fp = bdone + bofs[mat] + bp;
        int* const fq = bdone + bofs[mat] + bq;
        if (tid == 0 && round > 0) {
            const long long tw = clock64();
            if (!(flag_wait_geq(fp, round) && flag_wait_geq(fq, round))) atomicOr(err, DERR_TIMEOUT);
            atomicAdd(stats + 6, (unsigned long long)(clock64() - tw));
        }
        ++ntask;
        __syncthreads();
        auto grow = [&](int lr) -> int {
            const int r = (lr < 32 ? bp : bq) * 32 + (lr & 31);
            return r < d.rows ? r : -1;
        };
        const float absf = d.absfloor ? *d.absfloor : 0.0f;
        const long long t0 = clock64();
        bool rot_pair = false;

        // ---- 1. Gram matrix over ncols_dot columns
        {
            // staging: column scol of the chunk in rows srow0 + 4 j (j < 8: block bp,
            // else bq), so that a warp's load reads 32 consecutive columns of one row
            const int scol = tid & 63, srow0 = tid >> 6;
            const int rp0 = bp * 32 + srow0, rq0 = bq * 32 + srow0;
            float pre[16];
            auto load = [&](int c0) {
                const int c = c0 + scol;
                const bool cok = c < d.ncols_dot;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = (j < 8 ? rp0 : rq0) + 4 * (j & 7);
                    pre[j] = (cok && r < d.rows) ? __ldcg(d.A + (size_t)r * d.ld + c) : 0.0f;
                }
            };
            const int nch = (d.ncols_dot + JT_KC - 1) / JT_KC;
            if (nch > 0) load(0);
            // D f32, A and B tf32, both K-major, N = 64, M = 128
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const int colh = (warp >> 2) * 32;  // this warp's 32 of the 64 product columns
            const uint64_t sdesc0 = sw128_desc(smem_u32(rx));
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
            for (int i = 0; i < nch; ++i) {
                // tile i & 1: 128 rows x 64 k, two k atoms of 16 KB (rows 0..63 hi, 64..127 lo)
                unsigned char* S = rx + (i & 1) * 32768;
                unsigned char* Sa = S + (scol >> 5) * 16384;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float v = pre[j];
                    const float hi = tf32_rna(v);
                    const int row = srow0 + 4 * j;
                    *reinterpret_cast<float*>(Sa + sw128_off(row, scol & 31)) = hi;
                    *reinterpret_cast<float*>(Sa + sw128_off(row + 64, scol & 31)) = tf32_rna(v - hi);
                }
                if (i + 1 < nch) load((i + 1) * JT_KC);
                // the previous chunk's MMAs are done (its staging tile and product buffer are free)
                const bool mine = i > 0 ? mbar_wait(mb, (ncommit - 1) & 1u) : true;
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                if (!__syncthreads_and(mine ? 1 : 0)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (tid == 0) {
                    // descriptors advance by (byte offset >> 4) in their address field
                    const uint32_t dcol = tmem + (uint32_t)(i & 1) * 64;
                    const uint64_t sd = sdesc0 + (uint64_t)((i & 1) * (32768 >> 4));
#pragma unroll
                    for (int ks = 0; ks < JT_KC / 8; ++ks) {
                        const uint64_t da = sd + (uint64_t)(((ks >> 2) * 16384 + (ks & 3) * 32) >> 4);
                        mma_tf32(dcol, da, da, idesc, ks > 0 ? 1u : 0u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
                }
                ++ncommit;
                if (i > 0) {
                    const uint32_t prev = tmem + (uint32_t)((i - 1) & 1) * 64 + (uint32_t)colh + lane_off;
                    tmem_add16(prev, acc);
                    tmem_add16(prev + 16, acc + 16);
                }
            }
            if (ok && nch > 0) {
                const bool mine = mbar_wait(mb, (ncommit - 1) & 1u);
                if (!__syncthreads_and(mine ? 1 : 0)) {
                    ok = false;
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t last = tmem + (uint32_t)((nch - 1) & 1) * 64 + (uint32_t)colh + lane_off;
                    tmem_add16(last, acc);
                    tmem_add16(last + 16, acc + 16);
                }
            }
            if (ok) {
                // rows 0..63 of the product (hh) to G0, rows 64..127 (lh) to G1 (the
                // staging tiles are no longer read: every MMA is done)
                const int rho = 32 * (warp & 3) + lane;
                float* dst = rho < 64 ? G0 + rho * JPI_LDG : G1 + (rho - 64) * JPI_LDG;
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[colh + j] = acc[j];
                for (int e = tid; e < JPI_N * JPI_N; e += 256) Qt[(e >> 6) * JPI_LDQ + (e & 63)] = (e >> 6) == (e & 63) ? 1.0f : 0.0f;
                __syncthreads();
                // G = hh + lh + lh^T on the upper triangle and the diagonal
                for (int e = tid; e < JPI_N * JPI_N; e += 256) {
                    const int r = e >> 6, c = e & 63;
                    if (c < r) continue;
                    G0[r * JPI_LDG + c] += G1[r * JPI_LDG + c] + G1[c * JPI_LDG + r];
                }
                __syncthreads();
            }
        }

        // ---- 2. inner eigensolve (tests as in jacobi_pair_kernel)
        const float ueps = 1.1920928955078125e-7f;
        const float tin = fmaxf(tol * (1.0f / 64.0f), 16.0f * ueps);
        const long long t1 = clock64();
        if (ok) {
            if (tid == 0) {
                atomicAdd(stats + 0, 1ull);
                atomicAdd(stats + 2, (unsigned long long)(t1 - t0));
            }
            int mine = 0;
            for (int e = tid; e < JPI_N * JPI_N; e += 256) {
                const int p = e >> 6, q = e & 63;
                if (q <= p) continue;
                const float a = G0[p * JPI_LDG + p], b = G0[q * JPI_LDG + q], g = G0[p * JPI_LDG + q];
                if (g != 0.0f && g * g > tol * tol * a * b && fabsf(g) > absf) mine = 1;
            }
            rot_pair = __syncthreads_or(mine) != 0;
        }
        if (ok && rot_pair) {
            unsigned nrot = 0;
            const int inner = jpi_solve<float>(G0, G1, Qt, jr, tin, absf, inner_max, nrot);
            if (nrot) atomicAdd(rots + mat, (unsigned long long)nrot);
            const long long t2 = clock64();
            if (tid == 0) {
                rotated[mat] = 1;
                atomicAdd(stats + 1, 1ull);
                atomicAdd(stats + 3, (unsigned long long)(t2 - t1));
                atomicAdd(stats + 5, (unsigned long long)inner);
            }

            // ---- 3. Y <- Qt Y over ncols_rot columns, as D = Y_c^T Qt^T
            // hi and lo of Qt into region Q: B operand, row n = output row, k = row
            // of Y, K-major with two 32-wide k atoms of 64 rows (8 KB each)
            for (int e = tid; e < JPI_N * JPI_N; e += 256) {
                const int r = e >> 6, k = e & 63;
                const float v = Qt[r * JPI_LDQ + k];
                const float hi = tf32_rna(v);
                const uint32_t o = (uint32_t)(k >> 5) * 8192 + sw128_off(r, k & 31);
                *reinterpret_cast<float*>(rq + o) = hi;
                *reinterpret_cast<float*>(rq + 16384 + o) = tf32_rna(v - hi);
            }
            // staging of Y_c^T (A operand, 128 rows c x 64 k, hi at X, lo at X + 32 KB,
            // two k atoms of 16 KB): warp w takes 32 tiles of 8 columns x 4 rows, lane
            // l the entry (column 8 cb + (l & 7), row 4 kb + (l >> 3)); a warp's load
            // reads four 32-byte segments and its stores hit 32 distinct banks
            // (tile j of warp w: id = 32 w + j, cb = id & 15, kb = id >> 4 = 2 w + (j >> 4))
            const int cl = lane & 7, kl = lane >> 3;
            const int gy0 = grow(8 * warp + kl), gy1 = grow(8 * warp + 4 + kl);
            const float* yrow0 = gy0 >= 0 ? d.A + (size_t)gy0 * d.ld : nullptr;
            const float* yrow1 = gy1 >= 0 ? d.A + (size_t)gy1 * d.ld : nullptr;
            float pre[32];
            auto load = [&](int c0) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = c0 + 8 * (j & 15) + cl;
                    const float* rp = j < 16 ? yrow0 : yrow1;
                    pre[j] = (rp && c < d.ncols_rot) ? __ldcg(rp + c) : 0.0f;
                }
            };
            const int nch = (d.ncols_rot + JT_NC - 1) / JT_NC;
            // D f32, A and B tf32, both K-major, N = 64, M = 128
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint64_t adesc = sw128_desc(smem_u32(rx)), bdesc = sw128_desc(smem_u32(rq));
            const int ccol = 32 * (warp & 3) + lane;  // the column of the chunk this thread stores
            const int n0 = 32 * (warp >> 2);          // and its 32 rows n0 .. n0 + 31 (block bp or bq)
            const int gblk = (n0 == 0 ? bp : bq) * 32;
            const int nvalid = min(32, d.rows - gblk);  // rows of the block inside the matrix
            // chunk ci's product (tensor-memory buffer ci & 1, columns 64 (ci & 1) ..) to
            // global memory: two halves of 16 rows through registers
            auto drain = [&](int ci) {
                const int col = ci * JT_NC + ccol;
                float* out = d.A + (size_t)gblk * d.ld + col;
                const uint32_t tb = tmem + (uint32_t)((ci & 1) * 64);
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint32_t v[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                        : "r"(tb + (uint32_t)(n0 + 16 * hf) + lane_off));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (col < d.ncols_rot) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (16 * hf + j < nvalid) out[(size_t)(16 * hf + j) * d.ld] = __uint_as_float(v[j]);
                    }
                }
            };
            if (nch > 0) load(0);
            __syncthreads();  // Qt (FP32, region X) is read whole before region X is restaged
            for (int i = 0; i < nch; ++i) {
                if (i > 0) {
                    // chunk i - 1's MMAs are done: the staging tile is free and its product readable
                    const bool mine = mbar_wait(mb, (ncommit - 1) & 1u);
                    if (!__syncthreads_and(mine ? 1 : 0)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = 8 * (j & 15) + cl, k = 8 * warp + 4 * (j >> 4) + kl;
                    const float v = pre[j];
                    const float hi = tf32_rna(v);
                    const uint32_t o = (uint32_t)(k >> 5) * 16384 + sw128_off(c, k & 31);
                    *reinterpret_cast<float*>(rx + o) = hi;
                    *reinterpret_cast<float*>(rx + 32768 + o) = tf32_rna(v - hi);
                }
                if (i + 1 < nch) load((i + 1) * JT_NC);
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (tid == 0) {
                    const uint32_t dcol = tmem + (uint32_t)((i & 1) * 64);
#pragma unroll
                    for (int ks = 0; ks < JPI_N / 8; ++ks) {
                        const uint64_t ao = (uint64_t)(((ks >> 2) * 16384 + (ks & 3) * 32) >> 4);
                        const uint64_t bo = (uint64_t)(((ks >> 2) * 8192 + (ks & 3) * 32) >> 4);
                        mma_tf32(dcol, adesc + ao, bdesc + bo, idesc, ks > 0 ? 1u : 0u);
                        mma_tf32(dcol, adesc + ao, bdesc + bo + (16384 >> 4), idesc, 1u);
                        mma_tf32(dcol, adesc + ao + (32768 >> 4), bdesc + bo, idesc, 1u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
                }
                ++ncommit;
                // while chunk i runs, chunk i - 1 (done, waited above) goes out
                if (i > 0) drain(i - 1);
            }
            if (ok && nch > 0) {
                const bool mine = mbar_wait(mb, (ncommit - 1) & 1u);
                if (!__syncthreads_and(mine ? 1 : 0)) {
                    ok = false;
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    drain(nch - 1);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            if (tid == 0) atomicAdd(stats + 4, (unsigned long long)(clock64() - t2));
        }
        // every thread's stores of the rotated rows precede the flags
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            flag_publish(fp, round + 1);
            flag_publish(fq, round + 1);
        }
        if (!ok) break;  // uniform
    }  // task loop
    if (tid == 0) {
        atomicAdd(stats + 7, (unsigned long long)(clock64() - tlife));
        if (ntask > 0) atomicAdd(stats + 8, 1ull);
    }

    if (!ok) {
        // a wait gave up: latch the error and wait once more for the last commit
        // before the tensor memory is freed
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        if (ncommit > 0) (void)mbar_wait(mb, (ncommit - 1) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(JT_TMEM_COLS));
}

size_t jacobi_pair_tc_smem() { return (size_t)JT_X + JT_Q + 1024; }

int launch_jacobi_pair_tc_sweep(const JacobiDescT<float>* d, const int4* tasks, int ntasks, int* counter, int* bdone,
                                 const int* bofs, float tol, int inner, int* rotated, unsigned long long* rots,
                                 unsigned long long* stats, int* err, cudaStream_t s) {
    if (ntasks <= 0) return 0;
    const size_t smem = jacobi_pair_tc_smem();
    cudaFuncSetAttribute(jacobi_pair_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // two CTAs per SM need the largest shared-memory carveout
    cudaFuncSetAttribute(jacobi_pair_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_pair_tc_kernel, 256, smem);
    // The occupancy query answers one CTA per SM for every kernel that allocates
    // tensor memory.  This kernel's shared memory (two times 100 KB), registers
    // (two times 120 x 256) and tensor memory (two times 128 of 512 columns)
    // allow two, and the hardware runs two.  A CTA that is not resident only
    // starts once another has left, finds the queue empty and exits: tasks are
    // claimed by running CTAs only, so no wait depends on a CTA that has not started.
    const int grid = std::max(1, std::min(ntasks, nsm * std::max(per, 2)));
    jacobi_pair_tc_kernel<<<grid, 256, smem, s>>>(d, tasks, ntasks, counter, bdone, bofs, tol, inner, rotated, rots,
                                                  stats, err);
    return grid;
}

size_t gemm_tc_smem() { return 4 * (size_t)TC_TILE_BYTES + 1024; }

void launch_gemm_tc(const GemmDescT<float>* d_descs, const TileRef* d_tiles, int ntiles, int* err, cudaStream_t s) {
    if (ntiles <= 0) return;
    const size_t smem = gemm_tc_smem();
    cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gemm_tc_kernel<<<ntiles, 128, smem, s>>>(d_descs, d_tiles, ntiles, err);
}

// The persistent sweep's bounded flag wait on its own: one thread waits until
// *flag >= 1 for at most `limit` SM cycles and latches DERR_TIMEOUT in *err
// when it gives up.
__global__ void wait_selftest_kernel(const int* flag, long long limit, int* err) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !flag_wait_geq(flag, 1, limit)) atomicOr(err, DERR_TIMEOUT);
}

void launch_wait_selftest(const int* flag, long long limit, int* err, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(flag, limit, err);
}

}  // namespace amdd
