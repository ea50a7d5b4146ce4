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

size_t gemm_tc_smem() { return 4 * (size_t)TC_TILE_BYTES + 1024; }

void launch_gemm_tc(const GemmDescT<float>* d_descs, const TileRef* d_tiles, int ntiles, int* err, cudaStream_t s) {
    if (ntiles <= 0) return;
    const size_t smem = gemm_tc_smem();
    cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    gemm_tc_kernel<<<ntiles, 128, smem, s>>>(d_descs, d_tiles, ntiles, err);
}

}  // namespace amdd
