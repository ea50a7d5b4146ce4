// Host side of libamdd: the C ABI declared in amdd.h, the integer part of the
// setup (subdomain sets of Sec. 2.1 and the gather plans), the orchestration
// of the batched setup kernels (Eq. (Xi), Sec. 3.2, Eq. (tildeA), Eq. (Zi),
// Eq. (two_level_schwarz)) and the preconditioned conjugate gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include <map>
#include <mutex>
#include <tuple>

#include "amdd.h"
#include "amdd_internal.h"

using namespace amdd;

namespace {

struct Fail {
    amdd_status st;
};

inline void ck(cudaError_t e) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{e == cudaErrorMemoryAllocation ? AMDD_ERR_OOM : AMDD_ERR_CUDA};
    }
}

inline void require(bool ok) {
    if (!ok) throw Fail{AMDD_ERR_INVALID};
}

}  // namespace

// Kernel classes of the profile (one per kernel; the Jacobi solver split by use).
enum ProfK {
    PK_GATHER,
    PK_CHOL_DIAG,
    PK_CHOL_PANEL,
    PK_GEMM,
    PK_TRTRI,
    PK_JAC_SVD,
    PK_JAC_EIG,
    PK_JAC_F32,
    PK_TRIDIAG,
    PK_BISECT,
    PK_SMALL,
    PK_E_ASM,
    PK_SPMV,
    PK_GEMV,
    PK_GATHER_SCATTER,
    PK_PCG_VEC,
    // FP32 variants (mixed form)
    PK_GEMM_F32,
    PK_CHOL_DIAG_F32,
    PK_CHOL_PANEL_F32,
    PK_TRTRI_F32,
    PK_TRIDIAG_F32,
    PK_BISECT_F32,
    PK_GEMV_F32,
    PK_CSOLVE,
    PK_GMRES,
    PK_GEMM_TC,
    PK_SPLOCAL,
    PK_COUNT
};
static_assert(PK_COUNT == AMDD_PROF_CLASSES, "profile classes");
static const char* const kProfNames[PK_COUNT] = {
    "gather_values", "chol_diag", "chol_panel", "gemm_tiles", "trtri_diag", "jacobi_svd", "jacobi_eig", "jacobi_f32", "tridiag", "bisect",
    "small_dense", "e_offdiag", "spmv", "gemv_rows", "gather_scatter", "pcg_vectors",
    "gemm_tiles_f32", "chol_diag_f32", "chol_panel_f32", "trtri_diag_f32", "tridiag_f32", "bisect_f32",
    "gemv_rows_f32", "coarse_solve", "gmres_vectors", "gemm_tc_f32", "sparse_local"};

// class of a kernel in element type T (FP32 variants have their own classes)
template <typename T>
constexpr int pk(int k64, int k32) {
    return std::is_same<T, float>::value ? k32 : k64;
}

struct ProfState {
    bool on = false;
    uint32_t mask = ~0u;  // classes timed
    int64_t launches[PK_COUNT] = {};
    double flops[PK_COUNT] = {};
    double bytes[PK_COUNT] = {};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PK_COUNT];
    // events are created once and reused, so a profiled launch costs two
    // cudaEventRecord calls on the host
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaEvent_t take() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void clear() {  // forget the records, keep the events
        for (int k = 0; k < PK_COUNT; ++k) {
            ev[k].clear();
            launches[k] = 0;
            flops[k] = 0.0;
            bytes[k] = 0.0;
        }
        used = 0;
    }
    void release() {
        clear();
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

struct amdd_handle {
    cudaStream_t s = nullptr;
    cudaStream_t s2 = nullptr;  // second stream of the setup (look-ahead of the blocked Cholesky)
    cudaEvent_t ev_panel = nullptr, ev_far = nullptr;
    // third and fourth streams: the speculative coarse factorisation (tau > 1)
    cudaStream_t s3 = nullptr, s4 = nullptr;
    cudaEvent_t ev_panel3 = nullptr, ev_far3 = nullptr, ev_spec_in = nullptr, ev_spec_done = nullptr;
    ProfState prof;
    int64_t n = 0, nnz = 0;
    int N = 0, overlap = 0;
    double tau = 0.0, eps = 0.0;
    int max_sweeps = 60;
    int spmv_group = 4;
    // copy of A
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    // per-subdomain sizes
    std::vector<int32_t> nI, nG, nD, ni, nt, p;
    std::vector<int64_t> off_om, off_sq, off_zt, off_I, coff;
    int64_t sum_ni = 0, sum_sq = 0, sum_nI = 0, sum_nt = 0, nC = 0, sum_zt = 0;
    int max_ni = 0, max_nt = 0;
    int64_t apply_tri_elems = 0;  // sum_i ni (ni + 1): elements read by the two local triangular products
    // persistent device data of the apply
    int32_t* d_omega = nullptr;
    double* d_Y = nullptr;
    double* d_Yt = nullptr;
    double* d_Zt = nullptr;
    double* d_YE = nullptr;
    double* d_YEt = nullptr;
    GemvDesc* d_gv_l1 = nullptr;
    GemvDesc* d_gv_l2 = nullptr;
    GemvDesc* d_gv_c = nullptr;
    int32_t *d_rd_c = nullptr, *d_rl_c = nullptr;
    // coarse prolongation zc = Z e as row GEMVs over Z_i = Zt_i^T (nI x p_i)
    double* d_Zr = nullptr;
    double* d_zc = nullptr;
    GemvDesc* d_gv_zp = nullptr;
    int32_t *d_rd_zp = nullptr, *d_rl_zp = nullptr;
    int64_t n_zp = 0;
    std::vector<GemvDesc> gv_zp_h;  // host copy (the batched path rebinds x / y)
    int32_t *d_g4_desc = nullptr, *d_g4_row = nullptr;  // row groups (one warp each) of the local products
    int64_t n_g4 = 0;
    int32_t *d_order_g = nullptr, *d_own_sub = nullptr, *d_own_a = nullptr, *d_sc_idx = nullptr;
    int32_t *d_nI = nullptr, *d_p = nullptr;
    int64_t *d_sc_ptr = nullptr, *d_zt_off = nullptr, *d_coff = nullptr;
    double *d_rloc = nullptr, *d_tloc = nullptr, *d_yloc = nullptr;
    // mixed form: FP32 local factors and local work vectors
    int precision = 0;
    float *d_Y32 = nullptr, *d_Yt32 = nullptr;
    float *d_rloc32 = nullptr, *d_tloc32 = nullptr, *d_yloc32 = nullptr;
    GemvDescT<float>* d_gv_l1_32 = nullptr;
    GemvDescT<float>* d_gv_l2_32 = nullptr;
    double *d_c = nullptr, *d_e = nullptr, *d_ctmp = nullptr;
    // coarse solve: L_E (d_YE), L_E^T (d_YEt), inverses of its diagonal blocks
    double *d_Yd = nullptr, *d_Ydt = nullptr;
    int cSB = 0, cK = 0, coop_blocks = 0;
    double csolve_flops = 0.0, csolve_bytes = 0.0;
    std::vector<int> env_row;     // first non-zero column of each row of E (and L_E)
    std::vector<int> env_colend;  // one past the last non-zero row of each column of L_E
    int* d_env_row = nullptr;
    int32_t* d_cperm = nullptr;  // factorisation order of the coarse unknowns (NULL: subdomain order)
    double *d_cF = nullptr, *d_cG = nullptr;  // folded coarse solve (CoarseSolveArgs::F, G), NULL: not folded
    int *d_cfw0 = nullptr, *d_cgw1 = nullptr;
    int cFW = 0;
    double *d_cp = nullptr, *d_ep = nullptr;  // coarse vectors in that order (MAXB vectors)
    int* d_env_colend = nullptr;
    // eigenvectors of partial selections: 0 dense Jacobi, 1 LOBPCG from random
    // rows, 2 LOBPCG from the learned proposal
    int eig_solver = 0, keep_prop = 0;
    int n_robust = 0;  // subdomains whose Schur complement took the robust form (step 5b)
    bool diag_basis = true;  // full selections use the basis diag(A_II)^{-1/2}
    amdd_proposal prop{};
    bool have_prop = false;
    std::vector<int> eig_iters;  // per subdomain: LOBPCG iterations, -1 dense path, -2 not partial
    int n_partial = 0, lob_subs = 0, lob_max = 0, lob_fallbacks = 0;
    int64_t lob_total = 0;
    // batched right-hand sides (up to MAXB per pass), allocated on first use
    int mb_cap = 0;
    double *d_m_rloc = nullptr, *d_m_tloc = nullptr, *d_m_yloc = nullptr;
    float *d_m_rloc32 = nullptr, *d_m_tloc32 = nullptr, *d_m_yloc32 = nullptr;
    double *d_m_c = nullptr, *d_m_ctmp = nullptr, *d_m_e = nullptr, *d_m_zc = nullptr;
    GemvDesc* d_m_gv_zp = nullptr;
    double *d_m_q = nullptr, *d_m_r = nullptr, *d_m_z = nullptr, *d_m_p = nullptr, *d_m_part = nullptr;
    PcgScal* d_m_sc = nullptr;
    void* d_m_gv_l1 = nullptr;  // GemvDescT<double or float> per subdomain, on the batched buffers
    void* d_m_gv_l2 = nullptr;
    GemvDesc* d_m_gv_c = nullptr;
    std::vector<const void*> lm1, lm2;  // per subdomain: L_i^{-1} and L_i^{-T} (FP64 or FP32)
    // kept for amdd_proposal_export: features and Krylov bases of the partial subdomains
    float* prop_feat = nullptr;
    double* prop_bt = nullptr;
    std::vector<int> prop_sub;
    std::vector<int64_t> prop_off_b;
    // deflated / restricted forms (Sec. 4.1), allocated on first use: position
    // in the local vectors of each unknown's own copy (owner order), and work
    // vectors in global order
    int32_t* d_own_idx = nullptr;
    double *d_zg = nullptr, *d_t = nullptr;
    // multilevel form: kept copy of E with its block pattern (CSR), the
    // second level and the counters of its inner solves
    int keep_E = 0;
    int64_t* d_E_rowptr = nullptr;
    int32_t* d_E_col = nullptr;
    double* d_E_val = nullptr;
    int64_t E_nnz = 0;
    amdd_handle* next = nullptr;
    int in_restart = 30, in_maxit = 100;
    double in_rtol = 1e-4;
    int64_t in_calls = 0, in_its = 0;
    int in_max = 0;
    // GMRES(m) work, allocated on first use for restart length gm_cap
    int gm_cap = 0;
    int64_t gm_ldv = 0;  // leading dimension of the Krylov vectors
    double *d_gm_V = nullptr, *d_gm_Zp = nullptr, *d_gm_wA = nullptr, *d_gm_wB = nullptr, *d_gm_part = nullptr;
    GmState* d_gm_st = nullptr;
    // PCG work vectors
    double *d_r = nullptr, *d_z = nullptr, *d_pv = nullptr, *d_q = nullptr, *d_part = nullptr;
    PcgScal* d_sc = nullptr;
    int* d_err = nullptr;
    int* d_chk = nullptr;  // flag of the non-finite input check
    // host results
    std::vector<double> sigma_h;  // singular values of X_i, descending, at off_om
    std::vector<double> lam_h;    // eigenvalues of eq. (Zi), descending, at off_I
    int sweeps_svd = 0, sweeps_eig = 0, sweeps_svd32 = 0, sweeps_eig32 = 0;
    int64_t rot_svd = 0, rot_eig = 0;
    double setup_ms = 0.0;
    std::vector<void*> allocs;
    // device bytes allocated by the setup (persistent + temporary; nothing is
    // freed before the setup ends, so the sum is its peak) and the budget
    size_t bytes_now = 0, bytes_peak = 0, mem_budget = 0;
    double tie_band = 1e-10;
    int n_tied = 0;  // eigenvalues with |lambda tau - 1| <= tie_band
    int n_below_one = 0;  // computed eigenvalues below 1 (the shift of the splitting)
    int64_t pair_stats[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // block-pair Jacobi: tasks, rotated, cycles of 3 phases, inner sweeps
    int use_graphs = 1;
    int autotune = 1;  // GEMM tile autotuner (process-wide table)
    int tensor_cores = 0;  // FP32 GEMMs on tcgen05 (3xTF32)
    // sparse local Cholesky factors (amdd_opts.local_solver): columns of each
    // factor in a nested-dissection order, used by the local solves when kept
    int local_solver = 0;
    int jacobi_inner = 1;  // inner sweeps per block-pair visit
    bool sparse_local = false;
    void* d_sl_val = nullptr;  // FP64 or FP32 as the local solves
    uint16_t* d_sl_row = nullptr;
    int32_t* d_sl_colptr = nullptr;
    int32_t* d_sl_perm = nullptr;
    SparseLocalDesc* d_sl_desc = nullptr;
    size_t sl_smem = 0;  // shared memory of the largest factor without its vectors
    int sl_nmax = 0;     // largest subdomain (vectors: nb x sl_nmax entries)
    int64_t sl_nnz = 0;
    // PCG iterations as a CUDA graph (amdd_opts.use_graphs): a device-side
    // while-loop over one iteration, built on the first solve of a tolerance
    cudaGraph_t pg_graph = nullptr;
    cudaGraphExec_t pg_exec = nullptr;
    cudaStream_t s_cap = nullptr;  // private stream the loop is captured on (the legacy stream cannot be)
    double pg_tol2 = -1.0;
    bool pg_failed = false;  // the runtime could not capture the loop: per-iteration launches
    double *d_px = nullptr, *d_alog = nullptr, *d_blog = nullptr;
    int* d_maxit = nullptr;
    int pg_cap = 0;
    int64_t graph_solves = 0;  // solves whose iterations ran as the graph
};

namespace {

// Counts the bytes against the handle's budget (amdd_opts.mem_budget): an
// allocation past it is AMDD_ERR_OOM before anything is allocated.
void account(amdd_handle* h, size_t bytes) {
    if (h->mem_budget && h->bytes_now + bytes > h->mem_budget) throw Fail{AMDD_ERR_OOM};
    h->bytes_now += bytes;
    h->bytes_peak = std::max(h->bytes_peak, h->bytes_now);
}

// Stream-ordered allocation owned by the handle (freed by amdd_destroy).
template <class T>
T* dnew(amdd_handle* h, size_t count) {
    void* p = nullptr;
    account(h, std::max<size_t>(count, 1) * sizeof(T));
    ck(cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), h->s));
    h->allocs.push_back(p);
    return static_cast<T*>(p);
}

// Records CUDA events around one launch of kernel class k on the handle's
// stream when profiling is on, and accounts its algorithmic flops / bytes.
struct PScope {
    amdd_handle* h;
    int k;
    cudaStream_t st;
    cudaEvent_t b = nullptr;
    PScope(amdd_handle* hh, int kk, double flops = 0.0, double bytes = 0.0, cudaStream_t stream = nullptr)
        : h(hh), k(kk), st(stream ? stream : hh->s) {
        if (!h->prof.on || !((h->prof.mask >> k) & 1u)) return;
        b = h->prof.take();
        if (!b) return;
        cudaEventRecord(b, st);
        h->prof.launches[k] += 1;
        h->prof.flops[k] += flops;
        h->prof.bytes[k] += bytes;
    }
    ~PScope() {
        if (!b) return;
        cudaEvent_t e = h->prof.take();
        if (!e) return;
        cudaEventRecord(e, st);
        h->prof.ev[k].push_back({b, e});
    }
};

// Setup-lifetime context: temporary device buffers and the host arrays that
// back asynchronous uploads are kept until the final synchronisation.
struct Ctx {
    amdd_handle* h;
    std::vector<void*> temps;
    std::vector<std::shared_ptr<void>> keep;
    size_t tbytes = 0;  // bytes of the temporaries
    explicit Ctx(amdd_handle* hh) : h(hh) {}
    ~Ctx() {
        // work on the other setup streams may still read temporaries (after an error)
        if (h->s2) cudaStreamSynchronize(h->s2);
        if (h->s3) cudaStreamSynchronize(h->s3);
        if (h->s4) cudaStreamSynchronize(h->s4);
        for (void* p : temps) cudaFreeAsync(p, h->s);
        h->bytes_now -= std::min(h->bytes_now, tbytes);
    }
    template <class T>
    T* tnew(size_t count) {
        void* p = nullptr;
        account(h, std::max<size_t>(count, 1) * sizeof(T));
        ck(cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), h->s));
        temps.push_back(p);
        tbytes += std::max<size_t>(count, 1) * sizeof(T);
        return static_cast<T*>(p);
    }
    template <class T>
    T* up(const std::vector<T>& v, bool persistent = false) {
        T* d = persistent ? dnew<T>(h, v.size()) : tnew<T>(v.size());
        if (!v.empty()) {
            auto copy = std::make_shared<std::vector<T>>(v);
            ck(cudaMemcpyAsync(d, copy->data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->s));
            keep.push_back(copy);
        }
        return d;
    }
};

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Output tiles of a batch of GEMMs for tile size `tile`.
template <typename T>
std::vector<TileRef> gemm_tiles(const std::vector<GemmDescT<T>>& ds, int tile) {
    std::vector<TileRef> tiles;
    for (int d = 0; d < (int)ds.size(); ++d) {
        const GemmDescT<T>& g = ds[d];
        if (g.m <= 0 || g.n <= 0) continue;
        const int tm = cdiv(g.m, tile), tn = cdiv(g.n, tile);
        for (int a = 0; a < tm; ++a)
            for (int b = 0; b < tn; ++b) {
                if (g.lower && b > a) continue;
                tiles.push_back({d, a, b});
            }
    }
    return tiles;
}

// 64 x 64 tiles unless that leaves fewer than two CTAs per SM; then 32 x 32.
constexpr int SMALL_LAUNCH_TILES = 2 * 152;
// A launch with fewer 32 x 32 tiles than this uses 16 x 16 tiles: with FP64 at
// two multiply-adds per clock per SM, a few large tiles leave most SMs idle and
// each tile's chain long.
constexpr int TINY_LAUNCH_TILES = 152 / 2;
// Smallest batch (in 128 x 128 output tiles) that takes the tensor-core GEMM.
constexpr int TC_MIN_TILES = 16;
// Largest dynamic shared memory of a sparse local solve (one subdomain's factor
// and one vector).
constexpr size_t SPARSE_LOCAL_SMEM_MAX = 200 * 1024;

// Process-wide autotuner of the GEMM tile (amdd_opts.autotune): per element
// type and size bucket (the batch's count of 64 x 64 output tiles and its
// largest k, each rounded up to a power of two) the tile size, 16, 32 or 64,
// that ran a batch of that bucket fastest.  It is measured once per bucket,
// with CUDA events on the handle's stream, on the first batch whose outputs
// may be written more than once (beta = 0 and no output overlapping an
// input); until then the launch-size rule decides.  Every tile size sums each
// output over k in the same order, so the choice changes the time and never
// the result.
struct TileTuner {
    std::mutex mu;
    std::map<std::tuple<int, int, int>, int> best;
    int64_t measured = 0;  // buckets measured in this process
};
TileTuner& tile_tuner() {
    static TileTuner t;
    return t;
}

inline int ceil_log2(int64_t v) {
    int b = 0;
    while ((int64_t{1} << b) < v) ++b;
    return b;
}

template <typename T>
bool rewritable(const std::vector<GemmDescT<T>>& ds) {
    for (const GemmDescT<T>& g : ds) {
        if (g.m <= 0 || g.n <= 0) continue;
        if (g.beta != T(0)) return false;
        const char* c0 = reinterpret_cast<const char*>(g.C);
        const char* c1 = reinterpret_cast<const char*>(g.C + (size_t)(g.m - 1) * g.ldc + g.n);
        const int64_t ar = g.ta ? g.k : g.m, ac = g.ta ? g.m : g.k;
        const int64_t br = g.tb ? g.n : g.k, bc = g.tb ? g.k : g.n;
        const char* a0 = reinterpret_cast<const char*>(g.A);
        const char* a1 = reinterpret_cast<const char*>(g.A + (size_t)(ar - 1) * g.lda + ac);
        const char* b0 = reinterpret_cast<const char*>(g.B);
        const char* b1 = reinterpret_cast<const char*>(g.B + (size_t)(br - 1) * g.ldb + bc);
        if ((c0 < a1 && a0 < c1) || (c0 < b1 && b0 < c1)) return false;
    }
    return true;
}

template <typename T>
void gemm(Ctx& C, const std::vector<GemmDescT<T>>& ds) {
    int tile = GEMM_T;
    std::vector<TileRef> tiles = gemm_tiles(ds, tile);
    if (tiles.empty()) return;
    const int heuristic = (int)tiles.size() >= SMALL_LAUNCH_TILES
                              ? 64
                              : ((int)gemm_tiles(ds, 32).size() >= TINY_LAUNCH_TILES ? 32 : 16);
    tile = heuristic;
    const GemmDescT<T>* dd = C.up(ds);
    if (C.h->autotune) {
        int kmax = 1;
        for (const GemmDescT<T>& g : ds) kmax = std::max(kmax, g.k);
        const auto key = std::make_tuple((int)sizeof(T), ceil_log2((int64_t)tiles.size()), ceil_log2(kmax));
        TileTuner& tt = tile_tuner();
        int found = 0;
        {
            std::lock_guard<std::mutex> lock(tt.mu);
            auto it = tt.best.find(key);
            if (it != tt.best.end()) found = it->second;
        }
        if (found) {
            tile = found;
        } else if (rewritable(ds)) {
            float best_ms = 0.0f;
            int best_tile = heuristic;
            cudaEvent_t e0, e1;
            ck(cudaEventCreate(&e0));
            ck(cudaEventCreate(&e1));
            for (int cand : {64, 32, 16}) {
                const std::vector<TileRef> tc = gemm_tiles(ds, cand);
                const TileRef* dtc = C.up(tc);
                launch_gemm<T>(dd, dtc, (int)tc.size(), cand, C.h->s);  // warm (first-launch costs)
                ck(cudaEventRecord(e0, C.h->s));
                launch_gemm<T>(dd, dtc, (int)tc.size(), cand, C.h->s);
                ck(cudaEventRecord(e1, C.h->s));
                ck(cudaEventSynchronize(e1));
                float ms = 0.0f;
                ck(cudaEventElapsedTime(&ms, e0, e1));
                if (cand == 64 || ms < best_ms) {
                    best_ms = ms;
                    best_tile = cand;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            tile = best_tile;
            std::lock_guard<std::mutex> lock(tt.mu);
            tt.best[key] = best_tile;
            tt.measured += 1;
        }
    }
    if (tile != GEMM_T) tiles = gemm_tiles(ds, tile);
    if constexpr (std::is_same<T, float>::value) {
        // the tensor-core path (amdd_opts.tensor_cores) for batches of at least
        // TC_MIN_TILES 128 x 128 output tiles
        if (C.h->tensor_cores) {
            std::vector<TileRef> tt = gemm_tiles(ds, TC_GEMM_TILE);
            if ((int)tt.size() >= TC_MIN_TILES) {
                double fl = 0.0;
                for (const GemmDescT<T>& g : ds) {
                    if (g.m <= 0 || g.n <= 0) continue;
                    const double m = g.m, n = g.n;
                    const double outs = g.lower ? (n <= m ? m * n - n * (n - 1) / 2 : m * (m + 1) / 2) : m * n;
                    fl += 2.0 * outs * g.k;
                }
                const TileRef* dtt = C.up(tt);
                PScope ps(C.h, PK_GEMM_TC, fl);
                launch_gemm_tc(dd, dtt, (int)tt.size(), C.h->d_err, C.h->s);
                return;
            }
        }
    }
    double fl = 0.0;
    for (const GemmDescT<T>& g : ds) {
        if (g.m <= 0 || g.n <= 0) continue;
        const double m = g.m, n = g.n;
        const double outs = g.lower ? (n <= m ? m * n - n * (n - 1) / 2 : m * (m + 1) / 2) : m * n;
        fl += 2.0 * outs * g.k;
    }
    const TileRef* dt = C.up(tiles);
    PScope ps(C.h, pk<T>(PK_GEMM, PK_GEMM_F32), fl);
    launch_gemm<T>(dd, dt, (int)tiles.size(), tile, C.h->s);
}

template <typename T>
GemmDescT<T> gd(const T* A, int lda, int ta, const T* B, int ldb, int tb, T* Cm, int ldc, int m, int n, int k,
                double alpha, double beta, int lower) {
    GemmDescT<T> g;
    g.A = A;
    g.B = B;
    g.C = Cm;
    g.m = m;
    g.n = n;
    g.k = k;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.ta = ta;
    g.tb = tb;
    g.lower = lower;
    g.kfrom_row = 0;
    g.alpha = (T)alpha;
    g.beta = (T)beta;
    return g;
}

// Blocked right-looking Cholesky of a batch of matrices (lower triangles),
// each stopped at its own column `stop` (the trailing block then holds the
// Schur complement of the factored leading block).
//
// `env` (optional, one entry per matrix, may be null) gives each row's first
// non-zero column (the envelope).  The Cholesky factor keeps the envelope of
// the matrix, so panel row tiles and trailing-update tiles whose rows have no
// entries in the current block column are zero throughout and are skipped.
//
// Look-ahead: the trailing update of step k is split into the next block
// column ("near", on the handle's stream, right after the panel) and the rest
// ("far", on a second stream).  The far update of step k runs while the
// diagonal block and panel of step k+1 are factored; the near update of step
// k+1 waits for it, since both write block column k+2.  The order of the
// updates of every entry is fixed, so results do not depend on timing.
template <typename T>
void chol_batched(Ctx& C, const std::vector<CholDescT<T>>& ds, const std::vector<const std::vector<int>*>& env = {}) {
    if (ds.empty()) return;
    amdd_handle* h = C.h;
    cudaStream_t sm = h->s, ss = h->s2;
    CholDescT<T>* dd = C.up(ds);
    int maxstop = 0;
    for (const auto& d : ds) maxstop = std::max(maxstop, d.stop);
    bool far_pending = false;  // a far update was issued on ss and not yet joined
    auto active_rows = [&](int d, int r_begin, int r_end, int kend) {
        const std::vector<int>* e = (d < (int)env.size()) ? env[d] : nullptr;
        if (!e) return true;
        for (int r = r_begin; r < r_end; ++r)
            if ((*e)[r] < kend) return true;
        return false;
    };
    // tiles of one GEMM descriptor whose row and column blocks are both active
    auto update_tiles = [&](int gi, const GemmDescT<T>& g, int d, int row_base, int col_base, int kend, int tile,
                            std::vector<TileRef>& out, double& fl) {
        const int tm = cdiv(g.m, tile), tn = cdiv(g.n, tile);
        std::vector<char> ar(tm), ac(tn);
        for (int a = 0; a < tm; ++a)
            ar[a] = active_rows(d, row_base + a * tile, std::min(row_base + (a + 1) * tile, row_base + g.m), kend);
        for (int b = 0; b < tn; ++b)
            ac[b] = active_rows(d, col_base + b * tile, std::min(col_base + (b + 1) * tile, col_base + g.n), kend);
        for (int a = 0; a < tm; ++a)
            for (int b = 0; b < tn; ++b)
                if (ar[a] && ac[b] && !(g.lower && b > a)) {
                    out.push_back({gi, a, b});
                    const double ri = std::min(tile, g.m - a * tile), ci = std::min(tile, g.n - b * tile);
                    const double outs = (g.lower && a == b) ? ri * (ri + 1) / 2 : ri * ci;
                    fl += 2.0 * outs * g.k;
                }
    };
    for (int k0 = 0; k0 < maxstop; k0 += CHOL_NB) {
        {
            double fl = 0.0;
            for (const auto& c : ds)
                if (k0 < c.stop) {
                    const double kb = std::min(k0 + CHOL_NB, c.stop) - k0;
                    fl += 2.0 * kb * kb * kb / 3.0;
                }
            PScope ps(h, pk<T>(PK_CHOL_DIAG, PK_CHOL_DIAG_F32), fl);
            launch_chol_diag<T>(dd, (int)ds.size(), k0, h->d_err, sm);
        }
        std::vector<PanelRef> pt;
        double pfl = 0.0;
        std::vector<GemmDescT<T>> gn, gf;  // near / far updates
        std::vector<int> gn_d, gf_d, gn_kend, gf_kend;
        int tiles64 = 0;
        for (int d = 0; d < (int)ds.size(); ++d) {
            const CholDescT<T>& c = ds[d];
            if (k0 >= c.stop) continue;
            const int kend = std::min(k0 + CHOL_NB, c.stop);
            const int rows = c.n - kend;
            if (rows <= 0) continue;
            const int kb = kend - k0;
            for (int rt = 0; rt < cdiv(rows, PANEL_ROWS); ++rt)
                if (active_rows(d, kend + rt * PANEL_ROWS, std::min(c.n, kend + (rt + 1) * PANEL_ROWS), kend)) {
                    pt.push_back({d, rt});
                    pfl += (double)std::min(PANEL_ROWS, rows - PANEL_ROWS * rt) * kb * (kb + 1);
                }
            const T* P = c.A + (size_t)kend * c.ld + k0;  // panel rows [kend, n)
            const int w = std::max(0, std::min(CHOL_NB, c.stop - kend));  // next block column
            if (w > 0) {
                gn.push_back(gd(P, c.ld, 0, P, c.ld, 1, c.A + (size_t)kend * c.ld + kend, c.ld, rows, w, kb, -1.0, 1.0,
                                1));
                gn_d.push_back(d);
                gn_kend.push_back(kend);
            }
            if (rows - w > 0) {
                const T* Pf = P + (size_t)w * c.ld;
                gf.push_back(gd(Pf, c.ld, 0, Pf, c.ld, 1, c.A + (size_t)(kend + w) * c.ld + kend + w, c.ld, rows - w,
                                rows - w, kb, -1.0, 1.0, 1));
                gf_d.push_back(d);
                gf_kend.push_back(kend);
                tiles64 += cdiv(rows - w, 64) * (cdiv(rows - w, 64) + 1) / 2;
            }
        }
        if (!pt.empty()) {
            const PanelRef* dpt = C.up(pt);
            PScope ps(h, pk<T>(PK_CHOL_PANEL, PK_CHOL_PANEL_F32), pfl);
            launch_chol_panel<T>(dd, dpt, (int)pt.size(), k0, sm);
        }
        // far update on the second stream, after this panel
        int tile = tiles64 < SMALL_LAUNCH_TILES ? 32 : 64;
        std::vector<TileRef> tf, tn;
        double ffl = 0.0, nfl = 0.0;
        auto far_tiles = [&]() {
            tf.clear();
            ffl = 0.0;
            for (int q = 0; q < (int)gf.size(); ++q) {
                const int kend = gf_kend[q];
                const int w = (int)(ds[gf_d[q]].n - kend) - gf[q].m;
                update_tiles(q, gf[q], gf_d[q], kend + w, kend + w, kend, tile, tf, ffl);
            }
        };
        far_tiles();
        if (tile == 32 && (int)tf.size() < TINY_LAUNCH_TILES) {
            tile = 16;
            far_tiles();
        }
        int ntile = 32;
        for (int q = 0; q < (int)gn.size(); ++q)
            update_tiles(q, gn[q], gn_d[q], gn_kend[q], gn_kend[q], gn_kend[q], ntile, tn, nfl);
        if ((int)tn.size() < TINY_LAUNCH_TILES) {
            ntile = 16;
            tn.clear();
            nfl = 0.0;
            for (int q = 0; q < (int)gn.size(); ++q)
                update_tiles(q, gn[q], gn_d[q], gn_kend[q], gn_kend[q], gn_kend[q], ntile, tn, nfl);
        }
        const GemmDescT<T>* dgf = tf.empty() ? nullptr : C.up(gf);
        const TileRef* dtf = tf.empty() ? nullptr : C.up(tf);
        const GemmDescT<T>* dgn = tn.empty() ? nullptr : C.up(gn);
        const TileRef* dtn = tn.empty() ? nullptr : C.up(tn);
        // the near update of this step writes block column k+1, which the far
        // update of the previous step also writes: join it first
        if (far_pending) {
            ck(cudaStreamWaitEvent(sm, h->ev_far, 0));
            far_pending = false;
        }
        if (!tf.empty()) {
            ck(cudaEventRecord(h->ev_panel, sm));
            ck(cudaStreamWaitEvent(ss, h->ev_panel, 0));
            {
                PScope ps(h, pk<T>(PK_GEMM, PK_GEMM_F32), ffl, 0.0, ss);
                launch_gemm<T>(dgf, dtf, (int)tf.size(), tile, ss);
            }
            ck(cudaEventRecord(h->ev_far, ss));
            far_pending = true;
        }
        if (!tn.empty()) {
            PScope ps(h, pk<T>(PK_GEMM, PK_GEMM_F32), nfl);
            launch_gemm<T>(dgn, dtn, (int)tn.size(), ntile, sm);
        }
    }
    if (far_pending) ck(cudaStreamWaitEvent(sm, h->ev_far, 0));
}

// Y = L^{-1} (lower triangular) for a batch, from the factors and the
// diagonal-block inverses left by chol_batched.
template <typename T>
void trtri_batched(Ctx& C, const std::vector<TrtriDescT<T>>& ds) {
    if (ds.empty()) return;
    amdd_handle* h = C.h;
    TrtriDescT<T>* dd = C.up(ds);
    int maxn = 0;
    for (const auto& d : ds) maxn = std::max(maxn, d.n);
    {
        PScope ps(h, PK_SMALL);
        launch_set_identity<T>(dd, (int)ds.size(), maxn, h->s);
    }
    for (int k0 = 0; k0 < maxn; k0 += CHOL_NB) {
        std::vector<ChunkRef> ch;
        std::vector<GemmDescT<T>> g;
        double fl = 0.0;
        for (int d = 0; d < (int)ds.size(); ++d) {
            const TrtriDescT<T>& t = ds[d];
            if (k0 >= t.n) continue;
            const int kend = std::min(k0 + CHOL_NB, t.n);
            for (int ct = 0; ct * 64 < kend; ++ct) ch.push_back({d, ct});
            fl += (double)kend * (kend - k0) * (kend - k0 + 1);
            if (kend < t.n)
                g.push_back(gd(t.L + (size_t)kend * t.ld + k0, t.ld, 0, t.Y + (size_t)k0 * t.ldy, t.ldy, 0,
                               t.Y + (size_t)kend * t.ldy, t.ldy, t.n - kend, kend, kend - k0, -1.0, 1.0, 0));
        }
        {
            const ChunkRef* dch = C.up(ch);
            PScope ps(h, pk<T>(PK_TRTRI, PK_TRTRI_F32), fl);
            launch_trtri_diag<T>(dd, dch, (int)ch.size(), k0, h->s);
        }
        gemm(C, g);
    }
}

template <typename T>
void transpose_batched(Ctx& C, const std::vector<const T*>& src, const std::vector<T*>& dst,
                       const std::vector<int>& n, const std::vector<int>& lds, const std::vector<int>& ldd) {
    if (src.empty()) return;
    int maxn = *std::max_element(n.begin(), n.end());
    auto a = C.up(src);
    auto b = C.up(dst);
    auto c = C.up(n);
    auto d = C.up(lds);
    auto e = C.up(ldd);
    PScope ps(C.h, PK_SMALL);
    launch_transpose<T>(a, b, c, d, e, (int)src.size(), maxn, C.h->s);
}

// Block-pair one-sided Jacobi (rows in global memory): the host runs the
// sweeps, each either as one launch per round over every matrix still
// rotating or, in FP32 with amdd_opts.tensor_cores, as one persistent launch
// of the kernel whose Gram matrices and rotations run on the tensor cores
// (its CTAs take the pairs in round order and start a pair once both of its
// row blocks have finished the previous round, so matrices of different
// sizes and consecutive rounds overlap), and drops a matrix after a sweep in
// which none of its block pairs needed a rotation (sweeps[m] then counts that sweep, as the row kernels
// do).  A matrix still rotating after max_sweeps keeps sweeps[m] = max_sweeps
// and, with report_noconv, latches DERR_EIG_NOCONV.
template <typename T>
void jacobi_pairs(Ctx& C, const std::vector<JacobiDescT<T>>& jd, const JacobiDescT<T>* djd, int max_sweeps, T tol,
                  int* sweeps, unsigned long long* rots, int report_noconv) {
    amdd_handle* h = C.h;
    const int nm = (int)jd.size();
    std::vector<int> nblk(nm), active;
    auto sw = std::make_shared<std::vector<int>>(nm, max_sweeps);
    for (int m = 0; m < nm; ++m) {
        const int b = cdiv(std::max(jd[m].rows, 1), JP_ROWS);
        nblk[m] = std::max(2, b + (b & 1));
        if (jd[m].rows >= 2)
            active.push_back(m);
        else
            (*sw)[m] = 1;
    }
    int* d_rot = C.tnew<int>(nm);
    std::vector<int> rot_h(nm);
    unsigned long long* d_st = C.tnew<unsigned long long>(9);
    ck(cudaMemsetAsync(d_st, 0, 9 * sizeof(unsigned long long), h->s));
    // FP32 on the tensor cores: one persistent launch per sweep, tasks in round
    // order, per-block round counters
    const bool tc_sweep = std::is_same<T, float>::value && h->tensor_cores;
    std::vector<int> bofs(nm + 1, 0);
    for (int m = 0; m < nm; ++m) bofs[m + 1] = bofs[m] + nblk[m];
    const int* d_bofs = tc_sweep ? C.up(bofs) : nullptr;
    int* d_flags = tc_sweep ? C.tnew<int>(bofs[nm] + 1) : nullptr;  // block counters, then the task counter
    for (int sweep = 0; sweep < max_sweeps && !active.empty(); ++sweep) {
        std::vector<int4> tasks;
        int maxb = 2;
        for (int m : active) maxb = std::max(maxb, nblk[m]);
        if (tc_sweep) {
            // within a round the largest matrices first: their chains of rounds are
            // the longest, the smaller matrices fill in behind them
            std::vector<int> order(active);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nblk[a] > nblk[b]; });
            for (int r = 0; r < maxb - 1; ++r)
                for (int m : order)
                    if (r < nblk[m] - 1)
                        for (int k = 0; k < nblk[m] / 2; ++k) tasks.push_back(make_int4(m, k, nblk[m], r));
        } else {
            for (int m : active)
                for (int k = 0; k < nblk[m] / 2; ++k) tasks.push_back(make_int4(m, k, nblk[m], 0));
        }
        const int4* dt = C.up(tasks);
        ck(cudaMemsetAsync(d_rot, 0, nm * sizeof(int), h->s));
        if constexpr (std::is_same<T, float>::value) {
            if (tc_sweep) {
                ck(cudaMemsetAsync(d_flags, 0, (bofs[nm] + 1) * sizeof(int), h->s));
                h->pair_stats[9] += launch_jacobi_pair_tc_sweep(djd, dt, (int)tasks.size(), d_flags + bofs[nm], d_flags,
                                                                d_bofs, tol, h->jacobi_inner, d_rot, rots, d_st, h->d_err,
                                                                h->s);
            }
        }
        if (!tc_sweep)
            for (int r = 0; r < maxb - 1; ++r)
                launch_jacobi_pair_round<T>(djd, dt, (int)tasks.size(), r, tol, h->jacobi_inner, d_rot, rots, d_st,
                                            h->s);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(rot_h.data(), d_rot, nm * sizeof(int), cudaMemcpyDeviceToHost, h->s));
        ck(cudaStreamSynchronize(h->s));
        std::vector<int> still;
        for (int m : active) {
            if (rot_h[m])
                still.push_back(m);
            else
                (*sw)[m] = sweep + 1;
        }
        active.swap(still);
    }
    C.keep.push_back(sw);
    ck(cudaMemcpyAsync(sweeps, sw->data(), nm * sizeof(int), cudaMemcpyHostToDevice, h->s));
    unsigned long long st[9];
    ck(cudaMemcpyAsync(st, d_st, sizeof(st), cudaMemcpyDeviceToHost, h->s));
    ck(cudaStreamSynchronize(h->s));
    for (int k = 0; k < 9; ++k) h->pair_stats[k] += (int64_t)st[k];
    if (!active.empty() && report_noconv) launch_or_flag(h->d_err, DERR_EIG_NOCONV, h->s);
}

// One-sided Jacobi on the rows of a batch: the shared-memory-resident block
// kernel when the two row blocks of the largest matrix fit, else the
// block-pair form with the rows in global memory.
template <typename T>
void run_jacobi(Ctx& C, const std::vector<JacobiDescT<T>>& jd, const JacobiDescT<T>* djd, int max_sweeps, T tol,
                int* sweeps, unsigned long long* rots, int report_noconv) {
    amdd_handle* h = C.h;
    size_t smem8 = 0, smem16 = 0;
    int maxr = 0;
    for (const auto& j : jd) {
        smem8 = std::max(smem8, jacobi_block_smem<T>(j.rows, j.ncols_rot, JAC_CLUSTER));
        smem16 = std::max(smem16, jacobi_block_smem<T>(j.rows, j.ncols_rot, 2 * JAC_CLUSTER));
        maxr = std::max(maxr, j.rows);
    }
    if (!launch_jacobi_block<T>(djd, (int)jd.size(), smem8, smem16, maxr, max_sweeps, tol, sweeps, rots, h->d_err,
                                report_noconv, h->s))
        jacobi_pairs<T>(C, jd, djd, max_sweeps, tol, sweeps, rots, report_noconv);
}

// FP32 stage of the Jacobi solvers.  For each R x L matrix A_b (FP64, lda),
// an FP32 one-sided Jacobi on the rows of [float(A_b) | I] accumulates
// rotations Q32 with Q32 A_b nearly row-orthogonal (to FP32 accuracy); Q32 is
// then made orthogonal to FP64 accuracy by Cholesky-QR (G = Q Q^T = L L^T,
// Q <- L^{-1} Q).  The caller applies Q in FP64 and finishes with FP64 sweeps,
// which then start from pairs that are orthogonal to ~1e-5 and converge in a
// few sweeps.  `floor` adds the absolute rotation floor eps32 * max row norm^2
// (used where only absolute accuracy of the rows is needed).
struct PrecondJob {
    const double* A;
    int R, L, lda;
    double* Q;  // R x R output
};

void fp32_precondition(Ctx& C, const std::vector<PrecondJob>& jobs, bool floor, int max_sweeps32, int* sweeps32,
                       unsigned long long* rots32) {
    amdd_handle* h = C.h;
    const int nb = (int)jobs.size();
    if (nb == 0) return;
    std::vector<int64_t> o32(nb + 1, 0), oR(nb + 1, 0), oQ(nb + 1, 0), oL(nb + 1, 0);
    int maxR = 1, maxL = 1;
    for (int b = 0; b < nb; ++b) {
        const int64_t R = jobs[b].R, L = jobs[b].L;
        o32[b + 1] = o32[b] + R * (L + R);
        oR[b + 1] = oR[b] + R;
        oQ[b + 1] = oQ[b] + R * R;
        oL[b + 1] = oL[b] + (int64_t)cdiv(R, CHOL_NB) * CHOL_NB * CHOL_NB;
        maxR = std::max<int>(maxR, (int)R);
        maxL = std::max<int>(maxL, (int)L);
    }
    float* m32 = C.tnew<float>(o32[nb]);
    float* n32 = C.tnew<float>(oR[nb]);
    float* f32 = C.tnew<float>(nb);
    double* Qraw = C.tnew<double>(oQ[nb]);
    double* G = C.tnew<double>(oQ[nb]);
    double* Y = C.tnew<double>(oQ[nb]);
    double* linv = C.tnew<double>(oL[nb]);
    std::vector<CvtDesc> cd(nb);
    std::vector<JacobiDescT<float>> jd(nb);
    for (int b = 0; b < nb; ++b) {
        const PrecondJob& j = jobs[b];
        cd[b] = {j.A, j.R, j.L, j.lda, m32 + o32[b], Qraw + oQ[b]};
        jd[b] = {m32 + o32[b], j.R, j.L + j.R, j.L, j.L + j.R, n32 + oR[b], floor ? f32 + b : nullptr};
    }
    const CvtDesc* dcd = C.up(cd);
    const JacobiDescT<float>* djd = C.up(jd);
    {
        PScope ps(h, PK_SMALL);
        launch_to_f32_with_identity(dcd, nb, maxR, h->s);
    }
    if (floor) {
        PScope ps(h, PK_SMALL);
        launch_row_maxnorm2<float>(djd, nb, std::numeric_limits<float>::epsilon(), f32, h->s);
    }
    {
        double fl = 0.0;  // one sweep's inner products (rotations add more; counted for the FP64 stage only)
        for (const auto& j : jobs) fl += (double)j.R * (j.R - 1) / 2 * 2.0 * j.L;
        PScope ps(h, PK_JAC_F32, fl);
        const float tol32 = 8.0f * std::sqrt((float)maxL) * std::numeric_limits<float>::epsilon();
        run_jacobi<float>(C, jd, djd, max_sweeps32, tol32, sweeps32, rots32, 0);
    }
    {
        PScope ps(h, PK_SMALL);
        launch_extract_q(dcd, nb, maxR, h->s);
    }
    // Cholesky-QR re-orthogonalisation in FP64
    std::vector<GemmDesc> g1, g2;
    std::vector<CholDesc> ch;
    std::vector<TrtriDesc> tr;
    for (int b = 0; b < nb; ++b) {
        const int R = jobs[b].R;
        double* q = Qraw + oQ[b];
        g1.push_back(gd(q, R, 0, q, R, 1, G + oQ[b], R, R, R, R, 1.0, 0.0, 1));
        ch.push_back({G + oQ[b], R, R, R, nullptr, linv + oL[b]});
        tr.push_back({G + oQ[b], Y + oQ[b], linv + oL[b], R, R, R});
        g2.push_back(gd(Y + oQ[b], R, 0, q, R, 0, jobs[b].Q, R, R, R, R, 1.0, 0.0, 0));
    }
    gemm(C, g1);
    chol_batched(C, ch);
    trtri_batched(C, tr);
    gemm(C, g2);
}

// true when v[0..cnt) holds only finite values (one read of v, one
// synchronisation of the handle's stream)
bool all_finite(amdd_handle* h, const double* v, int64_t cnt) {
    if (!h->d_chk) h->d_chk = dnew<int>(h, 1);
    ck(cudaMemsetAsync(h->d_chk, 0, sizeof(int), h->s));
    launch_nonfinite(v, cnt, h->d_chk, h->s);
    int f = 0;
    ck(cudaMemcpyAsync(&f, h->d_chk, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    ck(cudaStreamSynchronize(h->s));
    return f == 0;
}

int read_err(amdd_handle* h) {
    int e = 0;
    ck(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    ck(cudaStreamSynchronize(h->s));
    return e;
}

amdd_status err_status(int e) {
    if (e & DERR_NOT_SPD) return AMDD_ERR_NOT_SPD;
    if (e & DERR_EIG_NOCONV) return AMDD_ERR_EIG_NOCONV;
    if (e & DERR_TIMEOUT) return AMDD_ERR_TIMEOUT;
    if (e) return AMDD_ERR_CUDA;
    return AMDD_OK;
}

// Sec. 2.1: Omega_Gi = nodes at graph distance 1..ov from Omega_Ii (ascending)
// and Omega_Di = nodes at distance ov+1 (ascending), by breadth-first layers
// on the CSR graph.  `mark` (length n) is a scratch stamp array: entries equal
// to `stamp` are treated as already reached; on return every node of
// Omega_Ii, Omega_Gi and Omega_Di carries `stamp`.
void overlap_layers(const int64_t* rp, const int32_t* ci, const std::vector<int32_t>& I, int ov, int32_t stamp,
                    int32_t* mark, std::vector<int32_t>& G, std::vector<int32_t>& D) {
    for (int32_t g : I) mark[g] = stamp;
    std::vector<int32_t> frontier = I;
    G.clear();
    D.clear();
    for (int d = 1; d <= ov + 1; ++d) {
        std::vector<int32_t> nw;
        for (int32_t v : frontier)
            for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
                const int32_t c = ci[k];
                if (mark[c] != stamp) {
                    mark[c] = stamp;
                    nw.push_back(c);
                }
            }
        std::sort(nw.begin(), nw.end());
        if (d <= ov)
            G.insert(G.end(), nw.begin(), nw.end());
        else
            D = nw;
        frontier.swap(nw);
    }
    std::sort(G.begin(), G.end());
}

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------
// T is the precision of the local work (sets aside): double for the plain
// FP64 form, float for the mixed form (local factors, local solves, the SVD
// of X_i, the splitting and the eigensolve in FP32; E, its factor and PCG in
// FP64).
// ---------------------------------------------------------------------------
// Learned warm start and block LOBPCG for the eigenvectors of eq. (Zi)
// ---------------------------------------------------------------------------
// Small symmetric semi-definite matrices G_q (of either sign; m_q x m_q,
// row-major, leading dimension ld_q, at base + off_q) are diagonalised by
// one-sided Jacobi on the rows of [G_q | I]: the rotated rows of G_q become
// lambda_j w_j^T, so the row norms are |lambda_j|, the right half holds the
// eigenvectors w_j as rows and the dot product of the two halves gives the
// sign.  Returns, per matrix, the eigenvalues ascending
// (host) and the device offset of each eigenvector row in W.
template <typename T>
struct SmallEig {
    T* W = nullptr;                          // [G | I] work, rows of eigenvectors in the right half
    std::vector<int64_t> off;                // per matrix: offset of its m x 2m block in W
    std::vector<std::vector<int>> row;       // per matrix: row of the j-th smallest eigenvalue
    std::vector<std::vector<double>> val;    // per matrix: eigenvalues, ascending
};

template <typename T>
SmallEig<T> small_eig(Ctx& C, const T* base, const std::vector<int64_t>& goff, const std::vector<int>& m,
                      const std::vector<int>& ldg) {
    amdd_handle* h = C.h;
    const int nq = (int)m.size();
    SmallEig<T> out;
    out.off.assign(nq + 1, 0);
    int maxm = 1;
    for (int q = 0; q < nq; ++q) {
        out.off[q + 1] = out.off[q] + (int64_t)m[q] * 2 * m[q];
        maxm = std::max(maxm, m[q]);
    }
    out.W = C.tnew<T>(std::max<int64_t>(out.off[nq], 1));
    std::vector<int64_t> src, dst;
    std::vector<int32_t> len;
    std::vector<TrtriDescT<T>> idd(nq);
    std::vector<JacobiDescT<T>> jd(nq);
    T* nrm = C.tnew<T>(std::max<int64_t>(out.off[nq], 1));
    double* norms = C.tnew<double>(std::max<int64_t>(out.off[nq], 1));
    std::vector<double*> np(nq);
    int64_t nacc = 0;
    for (int q = 0; q < nq; ++q) {
        for (int r = 0; r < m[q]; ++r) {
            src.push_back(goff[q] + (int64_t)r * ldg[q]);
            dst.push_back(out.off[q] + (int64_t)r * 2 * m[q]);
            len.push_back(m[q]);
        }
        idd[q] = {nullptr, out.W + out.off[q] + m[q], nullptr, m[q], 0, 2 * m[q]};
        jd[q] = {out.W + out.off[q], m[q], 2 * m[q], m[q], 2 * m[q], nrm + nacc, nullptr};
        np[q] = norms + nacc;
        nacc += m[q];
    }
    {
        auto a = C.up(src);
        auto b = C.up(dst);
        auto c = C.up(len);
        auto di = C.up(idd);
        PScope ps(h, PK_SMALL);
        launch_gather_rows<T>(base, a, out.W, b, c, (int64_t)src.size(), h->s);
        launch_set_identity<T>(di, nq, maxm, h->s);
    }
    const JacobiDescT<T>* djd = C.up(jd);
    int* sw = C.tnew<int>(nq);
    unsigned long long* rots = C.tnew<unsigned long long>(nq);
    {
        PScope ps(h, PK_JAC_EIG);
        const T tol = (std::is_same<T, double>::value ? T(2) : T(8)) * std::sqrt((T)maxm) * std::numeric_limits<T>::epsilon();
        run_jacobi<T>(C, jd, djd, h->max_sweeps, tol, sw, rots, 0);
    }
    {
        auto dn = C.up(np);
        PScope ps(h, PK_SMALL);
        launch_rownorms<T>(djd, nq, dn, (T*)nullptr, 0.0, 0, h->s);
    }
    // signs: at convergence row j of the left half is lambda_j times row j of
    // the right half (a unit vector), so sign(lambda_j) is that of their dot
    // product (the row norm alone gives |lambda_j|)
    double* dots = C.tnew<double>(std::max<int64_t>(nacc, 1));
    {
        std::vector<int64_t> ro;
        std::vector<int32_t> rl;
        for (int q = 0; q < nq; ++q)
            for (int r = 0; r < m[q]; ++r) {
                ro.push_back(out.off[q] + (int64_t)r * 2 * m[q]);
                rl.push_back(m[q]);
            }
        auto a = C.up(ro);
        auto b = C.up(rl);
        PScope ps(h, PK_SMALL);
        launch_half_dots<T>(out.W, a, b, (int64_t)ro.size(), dots, h->s);
    }
    std::vector<double> hn(nacc), hd(nacc);
    ck(cudaMemcpyAsync(hn.data(), norms, nacc * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    ck(cudaMemcpyAsync(hd.data(), dots, nacc * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    ck(cudaStreamSynchronize(h->s));
    for (int64_t t = 0; t < nacc; ++t)
        if (hd[t] < 0.0) hn[t] = -hn[t];
    out.row.resize(nq);
    out.val.resize(nq);
    nacc = 0;
    for (int q = 0; q < nq; ++q) {
        std::vector<int> o(m[q]);
        std::iota(o.begin(), o.end(), 0);
        const double* v = hn.data() + nacc;
        std::stable_sort(o.begin(), o.end(), [&](int x, int y) { return v[x] < v[y]; });
        out.row[q] = o;
        out.val[q].resize(m[q]);
        for (int j = 0; j < m[q]; ++j) out.val[q][j] = v[o[j]];
        nacc += m[q];
    }
    return out;
}

// Orthonormal basis (rows) of the span of the rows of S_q (r_q rows of n_q
// entries): rows scaled to unit norm, then two passes of S <- diag(w^{-1/2})
// V^T S from the eigendecomposition G = S S^T = V diag(w) V^T.  The first
// pass drops the directions with w <= 1e-12 w_max (well above the rounding
// level ~ r u w_max of a Gram matrix, where the exact zeros of a rank-
// deficient S land); the second, on rows that are already nearly
// orthonormal, keeps only w > 1/2.  The result overwrites S_q; the new row
// counts are returned.
template <typename T>
std::vector<int> orth_rows(Ctx& C, T* S, const std::vector<int64_t>& soff, const std::vector<int>& r,
                           const std::vector<int>& n, int ld) {
    amdd_handle* h = C.h;
    const int nq = (int)r.size();
    std::vector<int> rr = r;
    {
        std::vector<ScaleDesc<T>> sd(nq);
        for (int q = 0; q < nq; ++q) sd[q] = {S + soff[q], ld, rr[q], n[q], nullptr};
        auto d = C.up(sd);
        PScope ps(h, PK_SMALL);
        launch_scale_rows<T>(d, nq, 1, h->s);
    }
    int maxr = 1;
    for (int q = 0; q < nq; ++q) maxr = std::max(maxr, rr[q]);
    std::vector<int64_t> goff(nq + 1, 0), voff(nq + 1, 0);
    for (int q = 0; q < nq; ++q) {
        goff[q + 1] = goff[q] + (int64_t)maxr * maxr;
        voff[q + 1] = voff[q] + (int64_t)maxr * ld;
    }
    T* G = C.tnew<T>(goff[nq]);
    T* V = C.tnew<T>(goff[nq]);
    T* tmp = C.tnew<T>(voff[nq]);
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<GemmDescT<T>> g(nq);
        std::vector<int> ldg(nq, maxr);
        for (int q = 0; q < nq; ++q)
            g[q] = gd<T>(S + soff[q], ld, 0, S + soff[q], ld, 1, G + goff[q], maxr, rr[q], rr[q], n[q], 1.0, 0.0, 0);
        gemm(C, g);
        SmallEig<T> e = small_eig<T>(C, G, std::vector<int64_t>(goff.begin(), goff.end() - 1), rr, ldg);
        // kept eigenvector rows, and the scale w^{-1/2} of each
        std::vector<int64_t> src, dst;
        std::vector<int32_t> len;
        std::vector<T> f;
        std::vector<int64_t> foff(nq + 1, 0);
        std::vector<int> keep(nq);
        for (int q = 0; q < nq; ++q) {
            const double wmax = e.val[q].empty() ? 0.0 : e.val[q].back();
            int k = 0;
            for (int j = rr[q] - 1; j >= 0; --j) {  // largest first
                const double w = e.val[q][j];
                const bool ok = pass == 0 ? (w > 1e-12 * wmax) : (w > 0.5);
                if (!ok) continue;
                src.push_back(e.off[q] + (int64_t)e.row[q][j] * 2 * rr[q] + rr[q]);
                dst.push_back(goff[q] + (int64_t)k * maxr);
                len.push_back(rr[q]);
                f.push_back((T)(1.0 / std::sqrt(w)));
                ++k;
            }
            keep[q] = k;
            foff[q + 1] = foff[q] + k;
        }
        {
            auto a = C.up(src);
            auto b = C.up(dst);
            auto c = C.up(len);
            PScope ps(h, PK_SMALL);
            launch_gather_rows<T>(e.W, a, V, b, c, (int64_t)src.size(), h->s);
        }
        std::vector<GemmDescT<T>> g2(nq);
        for (int q = 0; q < nq; ++q)
            g2[q] = gd<T>(V + goff[q], maxr, 0, S + soff[q], ld, 0, tmp + voff[q], ld, keep[q], n[q], rr[q], 1.0, 0.0, 0);
        gemm(C, g2);
        const T* df = C.up(f);
        std::vector<ScaleDesc<T>> sd(nq);
        std::vector<int64_t> src2, dst2;
        std::vector<int32_t> len2;
        for (int q = 0; q < nq; ++q) {
            sd[q] = {tmp + voff[q], ld, keep[q], n[q], df + foff[q]};
            for (int j = 0; j < keep[q]; ++j) {
                src2.push_back(voff[q] + (int64_t)j * ld);
                dst2.push_back(soff[q] + (int64_t)j * ld);
                len2.push_back(n[q]);
            }
        }
        {
            auto d = C.up(sd);
            auto a = C.up(src2);
            auto b = C.up(dst2);
            auto c = C.up(len2);
            PScope ps(h, PK_SMALL);
            launch_scale_rows<T>(d, nq, 0, h->s);
            launch_gather_rows<T>(tmp, a, S, b, c, (int64_t)src2.size(), h->s);
        }
        rr = keep;
    }
    return rr;
}

// An operator applied to blocks of rows: out_q = in_q T_q^T for every matrix
// q with rows[q] > 0 (in_q, out_q at q * stride, leading dimension ld).
template <typename T>
using RowsOp = std::function<void(const T* in, T* out, int ld, int64_t stride, const std::vector<int>& rows)>;

// Block LOBPCG (Knyazev 2001, no preconditioner) for the p_q smallest
// eigenpairs of the symmetric T_q (n_q x n_q at Tm + toff[q], leading
// dimension ldt_q, or applied by op when op is given), block size k_q, from
// the initial rows X0_q (k_q x n_q at X0 + xoff[q], leading dimension n_q;
// overwritten).  Vectors are rows.  Per iteration: residual rows
// R = T X - diag(theta) X; stop when every wanted residual norm is
// <= tol + tol_rel |theta_j| + tol_max max_j |theta_j|; otherwise
// Rayleigh-Ritz on the orthonormalised rows of [X; R; P] and
// P = X_new - (X_new X^T) X.  With a threshold sel (not NaN) only the pairs
// with theta < sel are wanted: see the selection mode below.  On return the
// first p_q rows of X0_q are the Ritz vectors and theta_out[q] the Ritz
// values; iters[q] counts the iterations and ok[q] the convergence (2: the
// block holds fewer than all wanted pairs).
template <typename T>
void lobpcg_rows(Ctx& C, const T* Tm, const std::vector<int64_t>& toff, const std::vector<int>& ldt, T* X0,
                 const std::vector<int64_t>& xoff, const std::vector<int>& n, const std::vector<int>& k,
                 const std::vector<int>& p, double tol, int maxit, std::vector<int>& iters, std::vector<char>& ok,
                 std::vector<std::vector<double>>& theta_out, const RowsOp<T>* op = nullptr, double tol_rel = 0.0,
                 double tol_max = 0.0, double sel = std::numeric_limits<double>::quiet_NaN()) {
    amdd_handle* h = C.h;
    const int nq = (int)n.size();
    iters.assign(nq, 0);
    ok.assign(nq, 0);
    theta_out.assign(nq, {});
    if (nq == 0) return;
    int maxn = 1, maxk = 1;
    for (int q = 0; q < nq; ++q) {
        maxn = std::max(maxn, n[q]);
        maxk = std::max(maxk, k[q]);
    }
    const int ld = maxn;
    const int64_t blk = (int64_t)maxk * ld, blk3 = 3 * blk;
    T* X = C.tnew<T>(nq * blk);
    T* TX = C.tnew<T>(nq * blk);
    T* R = C.tnew<T>(nq * blk);
    T* P = C.tnew<T>(nq * blk);
    T* S = C.tnew<T>(nq * blk3);
    T* TS = C.tnew<T>(nq * blk3);
    T* G = C.tnew<T>((int64_t)nq * 9 * maxk * maxk);
    T* Cm = C.tnew<T>((int64_t)nq * 9 * maxk * maxk);
    T* M = C.tnew<T>((int64_t)nq * maxk * maxk);
    T* theta = C.tnew<T>((int64_t)nq * maxk);
    double* rn = C.tnew<double>((int64_t)nq * maxk);
    auto boff = [&](int q, int64_t b) { return (int64_t)q * b; };
    // rows of a small matrix (from SmallEig) -> dense rows at dst
    auto take_rows = [&](const SmallEig<T>& e, const std::vector<int>& mm, const std::vector<int>& cnt, T* dst,
                         int64_t dblk, int dld) {
        std::vector<int64_t> src, dsto;
        std::vector<int32_t> len;
        for (int q = 0; q < (int)mm.size(); ++q)
            for (int j = 0; j < cnt[q]; ++j) {
                src.push_back(e.off[q] + (int64_t)e.row[q][j] * 2 * mm[q] + mm[q]);
                dsto.push_back((int64_t)q * dblk + (int64_t)j * dld);
                len.push_back(mm[q]);
            }
        auto a = C.up(src);
        auto b = C.up(dsto);
        auto c = C.up(len);
        PScope ps(h, PK_SMALL);
        launch_gather_rows<T>(e.W, a, dst, b, c, (int64_t)src.size(), h->s);
    };
    auto copy_rows = [&](const T* from, int64_t fblk, T* to, int64_t tblk, const std::vector<int>& rows, int rfrom,
                         int rto) {
        std::vector<int64_t> src, dsto;
        std::vector<int32_t> len;
        for (int q = 0; q < nq; ++q)
            for (int j = 0; j < rows[q]; ++j) {
                src.push_back(boff(q, fblk) + (int64_t)(rfrom + j) * ld);
                dsto.push_back(boff(q, tblk) + (int64_t)(rto + j) * ld);
                len.push_back(n[q]);
            }
        if (src.empty()) return;
        auto a = C.up(src);
        auto b = C.up(dsto);
        auto c = C.up(len);
        PScope ps(h, PK_SMALL);
        launch_gather_rows<T>(from, a, to, b, c, (int64_t)src.size(), h->s);
    };
    // Rayleigh-Ritz on the orthonormal rows of S (rs rows): X <- first k Ritz rows
    auto rayleigh_ritz = [&](const std::vector<int>& rs) {
        std::vector<GemmDescT<T>> g1(nq), g2(nq);
        const int ldg = 3 * maxk;
        for (int q = 0; q < nq; ++q) {
            if (!op)
                g1[q] = gd<T>(S + boff(q, blk3), ld, 0, Tm + toff[q], ldt[q], 0, TS + boff(q, blk3), ld, rs[q], n[q],
                              n[q], 1.0, 0.0, 0);
            g2[q] = gd<T>(S + boff(q, blk3), ld, 0, TS + boff(q, blk3), ld, 1, G + (int64_t)q * 9 * maxk * maxk, ldg,
                          rs[q], rs[q], n[q], 1.0, 0.0, 0);
        }
        if (op)
            (*op)(S, TS, ld, blk3, rs);
        else
            gemm(C, g1);
        gemm(C, g2);
        std::vector<int64_t> go(nq);
        std::vector<int> lg(nq, ldg);
        for (int q = 0; q < nq; ++q) go[q] = (int64_t)q * 9 * maxk * maxk;
        SmallEig<T> e = small_eig<T>(C, G, go, rs, lg);
        std::vector<int> kk(nq);
        for (int q = 0; q < nq; ++q) kk[q] = std::min(k[q], rs[q]);
        take_rows(e, rs, kk, Cm, 9 * maxk * maxk, ldg);
        std::vector<GemmDescT<T>> g3(nq), g4(nq);
        std::vector<T> th((size_t)nq * maxk, T(0));
        for (int q = 0; q < nq; ++q) {
            g3[q] = gd<T>(Cm + (int64_t)q * 9 * maxk * maxk, ldg, 0, S + boff(q, blk3), ld, 0, X + boff(q, blk), ld,
                          kk[q], n[q], rs[q], 1.0, 0.0, 0);
            g4[q] = gd<T>(Cm + (int64_t)q * 9 * maxk * maxk, ldg, 0, TS + boff(q, blk3), ld, 0, TX + boff(q, blk), ld,
                          kk[q], n[q], rs[q], 1.0, 0.0, 0);
            for (int j = 0; j < kk[q]; ++j) th[(size_t)q * maxk + j] = (T)e.val[q][j];
            theta_out[q].assign(e.val[q].begin(), e.val[q].begin() + kk[q]);
        }
        gemm(C, g3);
        gemm(C, g4);
        ck(cudaMemcpyAsync(theta, th.data(), th.size() * sizeof(T), cudaMemcpyHostToDevice, h->s));
        ck(cudaStreamSynchronize(h->s));
        return kk;
    };
    // initial block: orthonormalise X0 and Rayleigh-Ritz on it
    {
        // the caller's X0 layout (xoff, leading dimension n_q) -> S
        std::vector<int64_t> src, dsto;
        std::vector<int32_t> len;
        for (int q = 0; q < nq; ++q)
            for (int j = 0; j < k[q]; ++j) {
                src.push_back(xoff[q] + (int64_t)j * n[q]);
                dsto.push_back(boff(q, blk3) + (int64_t)j * ld);
                len.push_back(n[q]);
            }
        auto a = C.up(src);
        auto b = C.up(dsto);
        auto c = C.up(len);
        PScope ps(h, PK_SMALL);
        launch_gather_rows<T>(X0, a, S, b, c, (int64_t)src.size(), h->s);
    }
    std::vector<int64_t> soff(nq);
    for (int q = 0; q < nq; ++q) soff[q] = boff(q, blk3);
    std::vector<int> rs = orth_rows<T>(C, S, soff, k, n, ld);
    std::vector<int> kx = rayleigh_ritz(rs);
    std::vector<char> haveP(nq, 0), live(nq, 1);
    for (int it = 0;; ++it) {
        // residuals of the live matrices
        std::vector<ResidDesc<T>> rd;
        std::vector<int> qs;
        for (int q = 0; q < nq; ++q)
            if (live[q]) {
                rd.push_back({X + boff(q, blk), TX + boff(q, blk), R + boff(q, blk), theta + (int64_t)q * maxk,
                              rn + (int64_t)q * maxk, ld, n[q], kx[q], std::min(p[q], kx[q])});
                qs.push_back(q);
            }
        if (qs.empty()) break;
        {
            auto d = C.up(rd);
            PScope ps(h, PK_SMALL);
            launch_residual_rows<T>(d, (int)rd.size(), h->s);
        }
        std::vector<double> hr((size_t)nq * maxk);
        ck(cudaMemcpyAsync(hr.data(), rn, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        ck(cudaStreamSynchronize(h->s));
        bool any = false;
        for (int q : qs) {
            double thmax = 0.0;
            for (double t : theta_out[q]) thmax = std::max(thmax, std::fabs(t));
            const double* rq = hr.data() + (size_t)q * maxk;
            const std::vector<double>& t = theta_out[q];
            const int w = std::min(p[q], kx[q]);
            auto small = [&](int j) { return rq[j] <= tol + tol_rel * std::fabs(t[j]) + tol_max * thmax; };
            bool conv = kx[q] >= p[q];
            if (!std::isnan(sel) && w > 0) {
                // selection mode: the wanted pairs are those with theta < sel.
                // Ritz values bound the smallest eigenvalues from above, so
                // theta_{w-1} < sel proves at least w of them: stop, the block is
                // too small (ok = 2).  Otherwise converge the pairs below sel and
                // require the first one above it to stay there within its
                // residual.
                if (t[w - 1] < sel) {
                    live[q] = 0;
                    ok[q] = 2;
                    iters[q] = it;
                    continue;
                }
                int js = 0;
                while (t[js] < sel) ++js;
                conv = t[js] - rq[js] >= sel;
                for (int j = 0; conv && j < js; ++j) conv = small(j);
            } else {
                for (int j = 0; conv && j < w; ++j) conv = small(j);
            }
            if (conv) {
                live[q] = 0;
                ok[q] = 1;
                iters[q] = it;
            } else if (it >= maxit) {
                live[q] = 0;
                iters[q] = it;
            } else {
                any = true;
            }
        }
        if (!any) break;
        // S = [X; R; P] for the live matrices (frozen ones keep a copy of X)
        std::vector<int> r3(nq);
        for (int q = 0; q < nq; ++q) r3[q] = live[q] ? kx[q] * (haveP[q] ? 3 : 2) : kx[q];
        {
            std::vector<int64_t> src, dsto;
            std::vector<int32_t> len;
            auto add = [&](int q, int rfrom, int rto, int cnt) {
                for (int j = 0; j < cnt; ++j) {
                    src.push_back(boff(q, blk) + (int64_t)(rfrom + j) * ld);
                    dsto.push_back(boff(q, blk3) + (int64_t)(rto + j) * ld);
                    len.push_back(n[q]);
                }
            };
            // three gathers (X, R, P) share the block layout of X
            for (int pass = 0; pass < 3; ++pass) {
                src.clear();
                dsto.clear();
                len.clear();
                const T* from = pass == 0 ? X : (pass == 1 ? R : P);
                for (int q = 0; q < nq; ++q) {
                    if (pass == 0) add(q, 0, 0, kx[q]);
                    if (pass == 1 && live[q]) add(q, 0, kx[q], kx[q]);
                    if (pass == 2 && live[q] && haveP[q]) add(q, 0, 2 * kx[q], kx[q]);
                }
                if (src.empty()) continue;
                auto a = C.up(src);
                auto b = C.up(dsto);
                auto c = C.up(len);
                PScope ps(h, PK_SMALL);
                launch_gather_rows<T>(from, a, S, b, c, (int64_t)src.size(), h->s);
            }
        }
        // keep the old X for the search direction
        copy_rows(X, blk, R, blk, kx, 0, 0);
        const std::vector<int> kold = kx;
        rs = orth_rows<T>(C, S, soff, r3, n, ld);
        kx = rayleigh_ritz(rs);
        // P = X_new - (X_new X_old^T) X_old (X_old in R)
        std::vector<GemmDescT<T>> g1, g2;
        for (int q = 0; q < nq; ++q) {
            if (!live[q]) continue;
            g1.push_back(gd<T>(X + boff(q, blk), ld, 0, R + boff(q, blk), ld, 1, M + (int64_t)q * maxk * maxk, maxk,
                               kx[q], kold[q], n[q], 1.0, 0.0, 0));
        }
        gemm(C, g1);
        copy_rows(X, blk, P, blk, kx, 0, 0);
        for (int q = 0; q < nq; ++q) {
            if (!live[q]) continue;
            g2.push_back(gd<T>(M + (int64_t)q * maxk * maxk, maxk, 0, R + boff(q, blk), ld, 0, P + boff(q, blk), ld,
                               kx[q], n[q], kold[q], -1.0, 1.0, 0));
            haveP[q] = 1;
        }
        gemm(C, g2);
    }
    // Ritz vectors back to the caller's layout
    std::vector<int64_t> src, dsto;
    std::vector<int32_t> len;
    for (int q = 0; q < nq; ++q)
        for (int j = 0; j < std::min(p[q], kx[q]); ++j) {
            src.push_back(boff(q, blk) + (int64_t)j * ld);
            dsto.push_back(xoff[q] + (int64_t)j * n[q]);
            len.push_back(n[q]);
        }
    auto a = C.up(src);
    auto b = C.up(dsto);
    auto c = C.up(len);
    PScope ps(h, PK_SMALL);
    launch_gather_rows<T>(X, a, X0, b, c, (int64_t)src.size(), h->s);
}

// Matrix-free eigensolve of eq. (Zi) (Sec. 3.2, eq. (invAii)), FP64.  With
// C = Sigma^{1/2} V^T the scaled rows of the SVD of X_i (step (2)) and
// C_I its Omega_Ii columns, eq. (invAii) restricted to Omega_Ii reads
//   (Abar_ii^{-1})_II = (1/delta) (I - C_I^T diag(1/(sigma + delta)) C_I),
// the inverse of the Schur complement S of Abar_ii onto Omega_Ii, so the
// wanted eigenpairs A_II u = lambda S u are the largest of the symmetric
//   K_i = L_A^T (Abar_ii^{-1})_II L_A,   u = L_A^{-T} y.
// Block LOBPCG on -K_i applies K_i to a block of rows X as four products,
// never forming Abar_ii, S or K_i:
//   Y = X L_A^T;  W = Y C_I^T;  Y -= W diag(1/(sigma+delta)) C_I;  X K_i = (1/delta) Y L_A.
// The two terms cancel to the working precision over delta, so the caller
// allows this path only for eps >= 2^-30.  The number of eigenvalues above
// 1/tau is not known in advance: LOBPCG runs in its selection mode (it
// converges the pairs above 1/tau and checks that the next one stays below),
// on a block that starts at max(16, nI/4) rows and doubles, restarted from
// its best rows, while a Ritz value proves the block too small (Ritz values
// are lower bounds of the largest eigenvalues) or the block did not
// converge; a block of nI rows spans everything (its Rayleigh-Ritz step is a
// dense eigensolve) and ends the search.  Returns per subdomain the computed
// lambda (descending: the selected ones and the first unselected one, or all)
// and their Ritz rows y (count x nI at rows[i]).
void mf_local_eigs(Ctx& C, amdd_handle* h, const double* X1, const std::vector<int64_t>& off_x, const double* sig,
                   const double* delta, double* Lb, std::vector<std::vector<double>>& lam,
                   std::vector<double*>& rows, std::vector<int>& its) {
    cudaStream_t s = h->s;
    const int N = h->N;
    lam.assign(N, {});
    rows.assign(N, nullptr);
    its.assign(N, -2);
    std::vector<double> dl(N);
    ck(cudaMemcpyAsync(dl.data(), delta, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> oc(N + 1, 0);
    int maxni = 1;
    for (int i = 0; i < N; ++i) {
        oc[i + 1] = oc[i] + (int64_t)h->ni[i] * h->nI[i];
        maxni = std::max(maxni, h->ni[i]);
    }
    double* Cc = C.tnew<double>(std::max<int64_t>(oc[N], 1));
    double* Bm = C.tnew<double>(std::max<int64_t>(oc[N], 1));
    {
        std::vector<MfPrepDesc> pd;
        std::vector<RowsDesc<double>> zu;
        for (int i = 0; i < N; ++i) {
            if (h->nI[i] == 0) continue;
            pd.push_back({X1 + off_x[i], h->nt[i], h->nG[i] + h->nD[i], h->ni[i], h->nI[i], sig + h->off_om[i],
                          delta + i, Cc + oc[i], Bm + oc[i]});
            // L_A (leading nI x nI block of the Cholesky factor of A_ii) enters
            // full GEMMs: clear the rest of its rows
            zu.push_back({Lb + h->off_sq[i], h->ni[i], 0, h->nI[i], h->nI[i], i});
        }
        if (pd.empty()) return;
        auto a = C.up(pd);
        auto b = C.up(zu);
        PScope ps(h, PK_SMALL);
        launch_mf_prepare(a, (int)pd.size(), maxni, s);
        launch_zero_upper<double>(b, (int)zu.size(), h->max_ni, s);
    }
    ck(cudaStreamSynchronize(s));
    std::vector<int> todo, kq(N, 0);
    double* pbase = nullptr;             // the previous round's block rows
    std::vector<int64_t> poff(N, 0);     // a subdomain's rows in it
    std::vector<int> prevn(N, 0);        // of which converged
    for (int i = 0; i < N; ++i)
        if (h->nI[i] > 0) {
            todo.push_back(i);
            kq[i] = std::min(h->nI[i], std::max(16, h->nI[i] / 4));
        }
    const double thr = 1.0 / h->tau;
    for (int round = 0; !todo.empty(); ++round) {
        const int nq = (int)todo.size();
        std::vector<int> n(nq), k(nq), want(nq), m(nq);
        std::vector<int64_t> xoff(nq + 1, 0), toff(nq, 0);
        std::vector<int> ldt(nq, 1);
        int maxk = 1;
        for (int q = 0; q < nq; ++q) {
            const int i = todo[q];
            n[q] = h->nI[i];
            k[q] = kq[i];
            want[q] = k[q] == n[q] ? n[q] : k[q] - std::max(2, k[q] / 8);
            m[q] = std::min(prevn[i], k[q]);
            xoff[q + 1] = xoff[q] + (int64_t)k[q] * n[q];
            maxk = std::max(maxk, k[q]);
        }
        double* X0 = C.tnew<double>(xoff[nq]);
        {
            std::vector<int64_t> src, dst;
            std::vector<int32_t> len;
            std::vector<RowsDesc<double>> rd(nq);
            for (int q = 0; q < nq; ++q) {
                const int i = todo[q];
                for (int j = 0; j < m[q]; ++j) {
                    src.push_back(poff[i] + (int64_t)j * n[q]);
                    dst.push_back(xoff[q] + (int64_t)j * n[q]);
                    len.push_back(n[q]);
                }
                rd[q] = {X0 + xoff[q], n[q], m[q], k[q], n[q], i};
            }
            if (!src.empty()) {
                auto a = C.up(src);
                auto b = C.up(dst);
                auto c = C.up(len);
                PScope ps(h, PK_SMALL);
                launch_gather_rows<double>(pbase, a, X0, b, c, (int64_t)src.size(), s);
            }
            auto d = C.up(rd);
            PScope ps(h, PK_SMALL);
            launch_rng_rows<double>(d, nq, maxk, 0x3A7Full + 0x1000ull * (unsigned long long)round, s);
        }
        double* Ybuf = nullptr;
        double* Wbuf = nullptr;
        RowsOp<double> op = [&](const double* in, double* out, int ld, int64_t stride, const std::vector<int>& r) {
            const int64_t wstride = stride / ld * maxni;
            if (!Ybuf) {
                Ybuf = C.tnew<double>(nq * stride);
                Wbuf = C.tnew<double>(nq * wstride);
            }
            std::vector<GemmDesc> g1, g2, g3, g4;
            for (int q = 0; q < nq; ++q) {
                if (r[q] == 0) continue;
                const int i = todo[q], ni = h->ni[i], nI = n[q];
                const double* LA = Lb + h->off_sq[i];
                double* Y = Ybuf + q * stride;
                double* W = Wbuf + q * wstride;
                g1.push_back(gd(in + q * stride, ld, 0, LA, ni, 1, Y, ld, r[q], nI, nI, 1.0, 0.0, 0));
                g2.push_back(gd(Y, ld, 0, Cc + oc[i], nI, 1, W, maxni, r[q], ni, nI, 1.0, 0.0, 0));
                g3.push_back(gd(W, maxni, 0, Bm + oc[i], nI, 0, Y, ld, r[q], nI, ni, -1.0, 1.0, 0));
                g4.push_back(gd(Y, ld, 0, LA, ni, 0, out + q * stride, ld, r[q], nI, nI, -1.0 / dl[i], 0.0, 0));
            }
            gemm(C, g1);
            gemm(C, g2);
            gemm(C, g3);
            gemm(C, g4);
        };
        std::vector<int> iters;
        std::vector<char> ok;
        std::vector<std::vector<double>> th;
        // residuals to a floor set by the operator's own rounding: the
        // cancellation in eq. (invAii) leaves about u / eps per product
        // (K_i is invariant under a scaling of A, and sigma_1 / delta = 1 / eps)
        const double floor_abs = 1000.0 * 0x1p-53 / h->eps;
        lobpcg_rows<double>(C, nullptr, toff, ldt, X0, xoff, n, k, want, floor_abs, 100, iters, ok, th, &op, 1e-9, 0.0,
                            -thr);
        std::vector<int> next;
        for (int q = 0; q < nq; ++q) {
            const int i = todo[q];
            int got = std::min<int>(want[q], (int)th[q].size());
            const bool full = k[q] == n[q];
            const bool enough = ok[q] == 1;
            h->lob_max = std::max(h->lob_max, iters[q]);
            h->lob_total += iters[q];
            if (enough) {  // the selected pairs and the first unselected one
                int js = 0;
                while (js < got - 1 && -th[q][js] > thr) ++js;
                got = js + 1;
            }
            if (full || enough) {
                lam[i].resize(got);
                for (int j = 0; j < got; ++j) lam[i][j] = -th[q][j];
                rows[i] = X0 + xoff[q];
                its[i] = iters[q];
                ++h->lob_subs;
            } else {
                kq[i] = std::min(n[q], 2 * k[q]);
                poff[i] = xoff[q];
                prevn[i] = got;  // converged or not, the best rows found so far
                next.push_back(i);
            }
        }
        pbase = X0;
        todo = next;
    }
}

// MLP forward on n standardised feature rows X (n x 32): Q (n x 16 x 16,
// symmetrised).  Work: Z1, H1, Z2, H2, Y (n x 256 each).
void mlp_forward(Ctx& C, const float* Wb, const float* X, int n, float* work, float* Q) {
    amdd_handle* h = C.h;
    float* Z1 = work;
    float* H1 = Z1 + (size_t)n * PROP_NH;
    float* Z2 = H1 + (size_t)n * PROP_NH;
    float* H2 = Z2 + (size_t)n * PROP_NH;
    float* Y = H2 + (size_t)n * PROP_NH;
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(X, PROP_NF, 0, Wb + MLP_OFF_W1, PROP_NH, 0, Z1, PROP_NH, n, PROP_NH,
                                                    PROP_NF, 1.0, 0.0, 0)});
    launch_bias_act(Z1, Wb + MLP_OFF_B1, H1, n, PROP_NH, h->s);
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(H1, PROP_NH, 0, Wb + MLP_OFF_W2, PROP_NH, 0, Z2, PROP_NH, n, PROP_NH,
                                                    PROP_NH, 1.0, 0.0, 0)});
    launch_bias_act(Z2, Wb + MLP_OFF_B2, H2, n, PROP_NH, h->s);
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(H2, PROP_NH, 0, Wb + MLP_OFF_W3, PROP_NO, 0, Y, PROP_NO, n, PROP_NO,
                                                    PROP_NH, 1.0, 0.0, 0)});
    launch_bias_act(Y, Wb + MLP_OFF_B3, nullptr, n, PROP_NO, h->s);
    launch_symmetrise(Y, Q, n, h->s);
}

// Gradient of the mean squared Frobenius error (forward with Wb, work as in
// mlp_forward plus Q, dY, dH, dZ (n x 256) and n partial sums).
void mlp_backward(Ctx& C, const float* Wb, const float* X, const float* Qt, int n, float* work, float* grad,
                  float* loss) {
    amdd_handle* h = C.h;
    const size_t L = (size_t)n * PROP_NH;
    float* Z1 = work;
    float* H1 = Z1 + L;
    float* Z2 = H1 + L;
    float* H2 = Z2 + L;
    float* Q = H2 + 2 * L;  // after Y
    float* dY = Q + L;
    float* dH = dY + L;
    float* dZ = dH + L;
    float* part = dZ + L;
    mlp_forward(C, Wb, X, n, work, Q);
    launch_loss_grad(Q, Qt, dY, part, loss, n, h->s);
    // output layer
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(H2, PROP_NH, 1, dY, PROP_NO, 0, grad + MLP_OFF_W3, PROP_NO, PROP_NH,
                                                    PROP_NO, n, 1.0, 0.0, 0)});
    launch_colsum(dY, grad + MLP_OFF_B3, n, PROP_NO, h->s);
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(dY, PROP_NO, 0, Wb + MLP_OFF_W3, PROP_NO, 1, dH, PROP_NH, n, PROP_NH,
                                                    PROP_NO, 1.0, 0.0, 0)});
    launch_relu_back(dH, Z2, dZ, n * PROP_NH, h->s);
    // second hidden layer
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(H1, PROP_NH, 1, dZ, PROP_NH, 0, grad + MLP_OFF_W2, PROP_NH, PROP_NH,
                                                    PROP_NH, n, 1.0, 0.0, 0)});
    launch_colsum(dZ, grad + MLP_OFF_B2, n, PROP_NH, h->s);
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(dZ, PROP_NH, 0, Wb + MLP_OFF_W2, PROP_NH, 1, dH, PROP_NH, n, PROP_NH,
                                                    PROP_NH, 1.0, 0.0, 0)});
    launch_relu_back(dH, Z1, dZ, n * PROP_NH, h->s);
    // first layer
    gemm(C, std::vector<GemmDescT<float>>{gd<float>(X, PROP_NF, 1, dZ, PROP_NH, 0, grad + MLP_OFF_W1, PROP_NH, PROP_NF,
                                                    PROP_NH, n, 1.0, 0.0, 0)});
    launch_colsum(dZ, grad + MLP_OFF_B1, n, PROP_NH, h->s);
}

// Eigenvectors of the partial selections without the dense Jacobi: the
// features and Krylov bases of those subdomains (kept in the handle for
// amdd_proposal_export when asked), then, with eig_solver >= 1, block LOBPCG
// for the p_i eigenvectors of T_i with the smallest mu, started from random
// rows (eig_solver = 1) or from the learned proposal (eig_solver = 2: the MLP
// predicts the projector onto the selected space on the Krylov basis; its
// leading eigenvectors B W give u, mapped to T's coordinates by w = L_A^T u,
// and random rows fill the block).  A result is accepted when every wanted
// residual is within the tolerance, the rows are orthonormal and the Ritz
// values agree with the bisection eigenvalues (a missed mode would show as a
// Ritz value above tau); its rows go to Wsel.  Returns the subdomains left to the dense path.
template <typename T>
std::vector<int> learned_eigvecs(Ctx& C, amdd_handle* h, const std::vector<int>& partial, const double* Araw, T* Lb,
                                 const T* TI, const std::vector<int64_t>& off_ti, T* Wsel) {
    constexpr bool f64 = std::is_same<T, double>::value;
    cudaStream_t s = h->s;
    const int np = (int)partial.size();
    std::vector<int64_t> off_b(np + 1, 0), off_w(np + 1, 0);
    for (int q = 0; q < np; ++q) {
        const int nIi = h->nI[partial[q]];
        off_b[q + 1] = off_b[q] + (int64_t)PROP_NB * nIi;
        off_w[q + 1] = off_w[q] + nIi;
    }
    const bool warm = h->eig_solver == 2 && h->have_prop;
    float* feat = nullptr;
    double* bt = nullptr;
    if (warm || h->keep_prop) {
        feat = C.tnew<float>((int64_t)np * PROP_NF);
        bt = C.tnew<double>(off_b[np]);
        double* wscr = C.tnew<double>(off_w[np]);
        std::vector<FeatDesc> fd(np);
        std::vector<KrylovDesc> kd(np);
        for (int q = 0; q < np; ++q) {
            const int i = partial[q], ni = h->ni[i];
            fd[q] = {Araw + h->off_sq[i], ni, ni, h->nI[i], h->nG[i], h->nD[i], h->p[i], h->tau, feat + (int64_t)q * PROP_NF};
            kd[q] = {Araw + h->off_sq[i], ni, h->nI[i], bt + off_b[q], wscr + off_w[q]};
        }
        auto dfd = C.up(fd);
        auto dkd = C.up(kd);
        PScope ps(h, PK_SMALL);
        launch_features(dfd, np, s);
        launch_krylov(dkd, np, s);
        if (h->keep_prop) {
            h->prop_feat = dnew<float>(h, (int64_t)np * PROP_NF);
            h->prop_bt = dnew<double>(h, off_b[np]);
            ck(cudaMemcpyAsync(h->prop_feat, feat, (size_t)np * PROP_NF * sizeof(float), cudaMemcpyDeviceToDevice, s));
            ck(cudaMemcpyAsync(h->prop_bt, bt, off_b[np] * sizeof(double), cudaMemcpyDeviceToDevice, s));
            h->prop_sub = partial;
            h->prop_off_b = off_b;
        }
    }
    if (h->eig_solver < 1) return partial;
    std::vector<int> n(np), k(np), p(np), m(np, 0), ldt(np);
    std::vector<int64_t> xoff(np + 1, 0), toff(np);
    int maxk = 1;
    for (int q = 0; q < np; ++q) {
        const int i = partial[q];
        n[q] = h->nI[i];
        p[q] = h->p[i];
        k[q] = std::min(n[q], p[q] + std::max(4, p[q] / 8));
        xoff[q + 1] = xoff[q] + (int64_t)k[q] * n[q];
        toff[q] = off_ti[i];
        ldt[q] = 2 * n[q];
        maxk = std::max(maxk, k[q]);
    }
    T* X0 = C.tnew<T>(xoff[np]);
    if (warm) {
        float* Xn = C.tnew<float>((int64_t)np * PROP_NF);
        launch_normalize_features(feat, h->prop.mean, h->prop.sd, Xn, np, s);
        float* work = C.tnew<float>((int64_t)5 * np * PROP_NH);
        float* Qh = C.tnew<float>((int64_t)np * PROP_NO);
        mlp_forward(C, h->prop.weights, Xn, np, work, Qh);
        std::vector<int64_t> go(np);
        std::vector<int> mm(np, PROP_NB), lg(np, PROP_NB);
        for (int q = 0; q < np; ++q) go[q] = (int64_t)q * PROP_NO;
        SmallEig<float> e = small_eig<float>(C, Qh, go, mm, lg);
        float* Wt = C.tnew<float>((int64_t)np * PROP_NO);
        std::vector<int64_t> src, dst;
        std::vector<int32_t> len;
        for (int q = 0; q < np; ++q) {
            m[q] = std::min(std::min(p[q], PROP_NB), k[q]);
            for (int j = 0; j < m[q]; ++j) {  // leading eigenvectors first
                src.push_back(e.off[q] + (int64_t)e.row[q][PROP_NB - 1 - j] * 2 * PROP_NB + PROP_NB);
                dst.push_back((int64_t)q * PROP_NO + (int64_t)j * PROP_NB);
                len.push_back(PROP_NB);
            }
        }
        {
            auto a = C.up(src);
            auto b = C.up(dst);
            auto c = C.up(len);
            PScope ps(h, PK_SMALL);
            launch_gather_rows<float>(e.W, a, Wt, b, c, (int64_t)src.size(), s);
        }
        const T* WtT;
        const T* BtT;
        if constexpr (f64) {
            double* w2 = C.tnew<double>((int64_t)np * PROP_NO);
            launch_convert<float, double>(Wt, w2, (int64_t)np * PROP_NO, s);
            WtT = w2;
            BtT = bt;
        } else {
            float* b2 = C.tnew<float>(off_b[np]);
            launch_convert<double, float>(bt, b2, off_b[np], s);
            WtT = Wt;
            BtT = b2;
        }
        T* U0 = C.tnew<T>(xoff[np]);
        std::vector<RowsDesc<T>> zu(np);
        int maxn = 1;
        std::vector<GemmDescT<T>> g1, g2;
        for (int q = 0; q < np; ++q) {
            const int i = partial[q], ni = h->ni[i];
            zu[q] = {Lb + h->off_sq[i], ni, 0, n[q], n[q], i};
            maxn = std::max(maxn, n[q]);
            if (m[q] == 0) continue;
            g1.push_back(gd<T>(WtT + (int64_t)q * PROP_NO, PROP_NB, 0, BtT + off_b[q], n[q], 0, U0 + xoff[q], n[q], m[q],
                               n[q], PROP_NB, 1.0, 0.0, 0));
            g2.push_back(gd<T>(U0 + xoff[q], n[q], 0, Lb + h->off_sq[i], ni, 0, X0 + xoff[q], n[q], m[q], n[q], n[q], 1.0,
                               0.0, 0));
        }
        {
            auto dz = C.up(zu);
            PScope ps(h, PK_SMALL);
            launch_zero_upper<T>(dz, np, maxn, s);
        }
        gemm(C, g1);
        gemm(C, g2);
    }
    {
        std::vector<RowsDesc<T>> rd(np);
        for (int q = 0; q < np; ++q) rd[q] = {X0 + xoff[q], n[q], m[q], k[q], n[q], partial[q]};
        auto d = C.up(rd);
        PScope ps(h, PK_SMALL);
        launch_rng_rows<T>(d, np, maxk, 0x5EEDull, s);
    }
    const double tol = f64 ? 1e-9 : 2e-4;
    std::vector<int> iters;
    std::vector<char> ok;
    std::vector<std::vector<double>> th;
    lobpcg_rows<T>(C, TI, toff, ldt, X0, xoff, n, k, p, tol, 60, iters, ok, th);
    // orthonormality of the returned rows (a rank-deficient block would make E singular)
    std::vector<int64_t> oo(np + 1, 0);
    for (int q = 0; q < np; ++q) oo[q + 1] = oo[q] + (int64_t)p[q] * p[q];
    T* Gx = C.tnew<T>(std::max<int64_t>(oo[np], 1));
    {
        std::vector<GemmDescT<T>> g;
        for (int q = 0; q < np; ++q)
            g.push_back(gd<T>(X0 + xoff[q], n[q], 0, X0 + xoff[q], n[q], 1, Gx + oo[q], p[q], p[q], p[q], n[q], 1.0, 0.0,
                              0));
        gemm(C, g);
    }
    std::vector<T> hg(oo[np]);
    ck(cudaMemcpyAsync(hg.data(), Gx, oo[np] * sizeof(T), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    const double otol = f64 ? 1e-8 : 1e-3;
    std::vector<int> dense;
    std::vector<int64_t> src, dst;
    std::vector<int32_t> len;
    for (int q = 0; q < np; ++q) {
        const int i = partial[q];
        bool accept = ok[q] && (int)th[q].size() >= p[q];
        for (int a = 0; accept && a < p[q]; ++a)
            for (int b = 0; b < p[q]; ++b)
                if (std::fabs((double)hg[oo[q] + (int64_t)a * p[q] + b] - (a == b ? 1.0 : 0.0)) > otol) accept = false;
        for (int j = 0; accept && j < p[q]; ++j) {
            const double lam = h->lam_h[h->off_I[i] + j];
            const double mu = std::isinf(lam) ? 0.0 : 1.0 / lam;
            if (std::fabs(th[q][j] - mu) > 1e-3 + 1e-3 * mu) accept = false;
        }
        if (!accept) {
            dense.push_back(i);
            ++h->lob_fallbacks;
            continue;
        }
        h->eig_iters[i] = iters[q];
        ++h->lob_subs;
        h->lob_max = std::max(h->lob_max, iters[q]);
        h->lob_total += iters[q];
        for (int j = 0; j < p[q]; ++j) {
            src.push_back(xoff[q] + (int64_t)j * n[q]);
            dst.push_back(h->off_zt[i] + (int64_t)j * n[q]);
            len.push_back(n[q]);
        }
    }
    if (!src.empty()) {
        auto a = C.up(src);
        auto b = C.up(dst);
        auto c = C.up(len);
        PScope ps(h, PK_SMALL);
        launch_gather_rows<T>(X0, a, Wsel, b, c, (int64_t)src.size(), s);
    }
    return dense;
}

// T: type of the local work (factors of A_ii, T = L_A^{-1} S L_A^{-T}, its
// eigensolve, Z_i).  TS: type of the splitting (SVD of X_i, Abar_ii and its
// Schur complement S).
// Reverse Cuthill-McKee order of a symmetric graph (adjacency lists): per
// connected component a pseudo-peripheral start (George and Liu: repeated
// breadth-first searches from a minimum-degree node of the deepest level),
// then breadth-first numbering with the unnumbered neighbours of each node by
// increasing degree; the whole sequence reversed.
std::vector<int32_t> rcm_order(const std::vector<std::vector<int32_t>>& nbr) {
    const int n = (int)nbr.size();
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<char> numbered(n, 0);
    std::vector<int> level(n, -1);
    auto deg = [&](int v) { return (int)nbr[v].size(); };
    // levels of the component of root among unnumbered nodes; returns the
    // depth and leaves the visited nodes in comp (levels reset on exit)
    std::vector<int32_t> comp, last;
    auto bfs = [&](int root) {
        comp.assign(1, root);
        level[root] = 0;
        int depth = 0;
        for (size_t head = 0; head < comp.size(); ++head) {
            const int v = comp[head];
            for (int w : nbr[v])
                if (level[w] < 0 && !numbered[w]) {
                    level[w] = level[v] + 1;
                    depth = std::max(depth, level[w]);
                    comp.push_back(w);
                }
        }
        last.clear();
        for (int v : comp)
            if (level[v] == depth) last.push_back(v);
        for (int v : comp) level[v] = -1;
        return depth;
    };
    for (int s0 = 0; s0 < n; ++s0) {
        if (numbered[s0]) continue;
        bfs(s0);
        int root = s0;
        for (int v : comp)
            if (deg(v) < deg(root)) root = v;
        int depth = bfs(root);
        for (int it = 0; it < 8; ++it) {
            int cand = last[0];
            for (int v : last)
                if (deg(v) < deg(cand)) cand = v;
            const int d2 = bfs(cand);
            if (d2 <= depth) break;
            root = cand;
            depth = d2;
        }
        const size_t start = order.size();
        order.push_back(root);
        numbered[root] = 1;
        std::vector<int32_t> nb;
        for (size_t head = start; head < order.size(); ++head) {
            const int v = order[head];
            nb.clear();
            for (int w : nbr[v])
                if (!numbered[w]) {
                    numbered[w] = 1;
                    nb.push_back(w);
                }
            std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg(a) < deg(b) || (deg(a) == deg(b) && a < b); });
            order.insert(order.end(), nb.begin(), nb.end());
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Sparse local factors (amdd_opts.local_solver): per subdomain the
// nested-dissection order of the local pattern and the column structure of its
// Cholesky factor (host, nd_factor_pattern); the permuted A_ii gathered dense on
// the device, factored by the batched dense Cholesky (entries outside the
// symbolic structure are rounding residues of exact zeros and are dropped), and
// its entries compacted into columns.  With local_solver = 2 (automatic) the
// factors are kept only when every subdomain's factor fits in shared memory and
// holds at most a quarter of its dense triangle; otherwise the dense inverse
// factors serve and nothing is kept.
template <typename T>
void build_sparse_local(Ctx& C, amdd_handle* h, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                        const std::vector<int32_t>& omega) {
    const int N = h->N;
    cudaStream_t s = h->s;
    std::vector<int32_t> perm_all(h->sum_ni), colptr_all;
    std::vector<uint16_t> rows_all;
    std::vector<int64_t> src_k, dst_p, ent_idx;
    std::vector<SparseLocalDesc> desc(N);
    std::vector<int32_t> stamp(h->n, -1), pos(h->n, -1);
    size_t smem_max = 0, smem_fixed = 0;
    int n_max = 0;
    int64_t nnz_tot = 0, dense_tot = 0;
    bool fits = true;
    for (int i = 0; i < N; ++i) {
        const int ni = h->ni[i];
        if (ni > 65535) {
            fits = false;
            break;
        }
        const int32_t* om = omega.data() + h->off_om[i];
        for (int a = 0; a < ni; ++a) {
            stamp[om[a]] = i;
            pos[om[a]] = a;
        }
        std::vector<int64_t> lrp(ni + 1, 0);
        std::vector<int32_t> lci;
        std::vector<int64_t> lk;  // global entry of each local entry
        for (int a = 0; a < ni; ++a) {
            const int32_t g = om[a];
            for (int64_t k = rp[g]; k < rp[g + 1]; ++k)
                if (stamp[ci[k]] == i) {
                    lci.push_back(pos[ci[k]]);
                    lk.push_back(k);
                }
            lrp[a + 1] = (int64_t)lci.size();
        }
        std::vector<int32_t> perm, colptr, rows;
        require(nd_factor_pattern(ni, lrp.data(), lci.data(), 16, perm, colptr, rows));
        std::vector<int32_t> iperm(ni);
        for (int k = 0; k < ni; ++k) iperm[perm[k]] = k;
        // the permuted matrix: local (a, b) goes to (iperm a, iperm b)
        for (int a = 0; a < ni; ++a)
            for (int64_t q = lrp[a]; q < lrp[a + 1]; ++q) {
                src_k.push_back(lk[q]);
                dst_p.push_back(h->off_sq[i] + (int64_t)iperm[a] * ni + iperm[lci[q]]);
            }
        const int nnz = colptr[ni];
        desc[i] = {ni, nnz, (int64_t)colptr_all.size(), nnz_tot, h->off_om[i]};
        colptr_all.insert(colptr_all.end(), colptr.begin(), colptr.end());
        for (int j = 0; j < ni; ++j)
            for (int q = colptr[j]; q < colptr[j + 1]; ++q) {
                const int r = rows[q];
                rows_all.push_back((uint16_t)r);
                const int64_t at = h->off_sq[i] + (int64_t)r * ni + j;  // lower triangle, row-major
                ent_idx.push_back(q == colptr[j] ? -at - 1 : at);        // diagonal: its reciprocal
            }
        std::copy(perm.begin(), perm.end(), perm_all.begin() + h->off_om[i]);
        nnz_tot += nnz;
        dense_tot += (int64_t)ni * (ni + 1) / 2;
        smem_fixed = std::max(smem_fixed, sparse_local_smem<T>(ni, nnz, 0));
        n_max = std::max(n_max, ni);
    }
    // a launch reserves the largest factor plus nb vectors of the largest
    // subdomain for every CTA, so the bound takes both maxima together
    smem_max = smem_fixed + (size_t)MAXB * n_max * sizeof(T);
    if (fits) fits = smem_max <= SPARSE_LOCAL_SMEM_MAX;
    if (h->local_solver == 2 && (!fits || 4 * nnz_tot > dense_tot)) return;  // automatic: dense
    require(fits);  // local_solver = 1 needs every factor in shared memory
    // numeric factorisation of the permuted matrices
    double* Ap = C.tnew<double>(h->sum_sq);
    ck(cudaMemsetAsync(Ap, 0, h->sum_sq * sizeof(double), s));
    {
        const int64_t* sk = C.up(src_k);
        const int64_t* dp = C.up(dst_p);
        PScope ps(h, PK_GATHER, 0.0, 32.0 * src_k.size());
        launch_gather_values(sk, dp, (int64_t)src_k.size(), h->val, Ap, s);
    }
    T* At = nullptr;
    if constexpr (std::is_same<T, double>::value) {
        At = Ap;
    } else {
        At = C.tnew<T>(h->sum_sq);
        launch_convert<double, T>(Ap, At, h->sum_sq, s);
    }
    std::vector<int64_t> off_lv(N + 1, 0);
    for (int i = 0; i < N; ++i) off_lv[i + 1] = off_lv[i] + (int64_t)cdiv(h->ni[i], CHOL_NB) * CHOL_NB * CHOL_NB;
    T* linv = C.tnew<T>(off_lv[N]);
    std::vector<CholDescT<T>> cd(N);
    for (int i = 0; i < N; ++i) cd[i] = {At + h->off_sq[i], h->ni[i], h->ni[i], h->ni[i], nullptr, linv + off_lv[i]};
    chol_batched(C, cd);
    // the factor's entries by column
    h->d_sl_val = dnew<T>(h, nnz_tot);
    {
        const int64_t* ei = C.up(ent_idx);
        PScope ps(h, PK_GATHER, 0.0, (8.0 + 2.0 * sizeof(T)) * nnz_tot);
        launch_gather_entries<T>(At, ei, static_cast<T*>(h->d_sl_val), nnz_tot, s);
    }
    h->d_sl_row = C.up(rows_all, true);
    h->d_sl_colptr = C.up(colptr_all, true);
    h->d_sl_perm = C.up(perm_all, true);
    h->d_sl_desc = C.up(desc, true);
    h->sl_smem = smem_fixed;
    h->sl_nmax = n_max;
    h->sl_nnz = nnz_tot;
    h->sparse_local = true;
}

template <typename T, typename TS>
void do_setup(amdd_handle* h, const amdd_csr* A, const int32_t* d_part) {
    constexpr bool f64 = std::is_same<T, double>::value;
    constexpr bool s64 = std::is_same<TS, double>::value;
    const int64_t n = A->n, nnz = A->nnz;
    const int N = h->N, ov = h->overlap;
    cudaStream_t s = h->s;
    Ctx C(h);

    h->d_err = dnew<int>(h, 1);
    ck(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    h->rowptr = dnew<int64_t>(h, n + 1);
    h->col = dnew<int32_t>(h, nnz);
    h->val = dnew<double>(h, nnz);
    ck(cudaMemcpyAsync(h->rowptr, A->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ck(cudaMemcpyAsync(h->col, A->colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    ck(cudaMemcpyAsync(h->val, A->val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    require(all_finite(h, h->val, nnz));  // a NaN or infinity in A: AMDD_ERR_INVALID

    // ---- host copies of the graph and the partition (integer setup, Sec. 2.1)
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> ci(nnz), part(n);
    ck(cudaMemcpyAsync(rp.data(), A->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(ci.data(), A->colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(part.data(), d_part, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    require(rp[0] == 0 && rp[n] == nnz);
    for (int64_t r = 0; r < n; ++r) require(rp[r] <= rp[r + 1]);
    for (int64_t k = 0; k < nnz; ++k) require(ci[k] >= 0 && ci[k] < n);
    std::vector<std::vector<int32_t>> Il(N);
    for (int64_t g = 0; g < n; ++g) {
        require(part[g] >= 0 && part[g] < N);
        Il[part[g]].push_back((int32_t)g);
    }
    for (int i = 0; i < N; ++i) require(!Il[i].empty());
    h->spmv_group = spmv_group_for(n, nnz);

    // ---- overlap Omega_Gi (distance 1..ov) and extension Omega_Di (ov+1)
    std::vector<std::vector<int32_t>> Gl(N), Dl(N);
    {
        std::vector<int32_t> mark(n, -1);
        for (int i = 0; i < N; ++i) overlap_layers(rp.data(), ci.data(), Il[i], ov, i, mark.data(), Gl[i], Dl[i]);
    }

    // ---- sizes and offsets
    h->nI.resize(N);
    h->nG.resize(N);
    h->nD.resize(N);
    h->ni.resize(N);
    h->nt.resize(N);
    h->off_om.assign(N + 1, 0);
    h->off_sq.assign(N + 1, 0);
    h->off_I.assign(N + 1, 0);
    std::vector<int64_t> off_x(N + 1, 0), off_m(N + 1, 0), off_ti(N + 1, 0), off_P(N + 1, 0), off_la(N + 1, 0),
        off_lm(N + 1, 0);
    for (int i = 0; i < N; ++i) {
        const int a = (int)Il[i].size(), b = (int)Gl[i].size(), c = (int)Dl[i].size();
        h->nI[i] = a;
        h->nG[i] = b;
        h->nD[i] = c;
        h->ni[i] = a + b;
        h->nt[i] = a + b + c;
        const int64_t ni = a + b, nt = a + b + c, nR = b + c;
        h->off_om[i + 1] = h->off_om[i] + ni;
        h->off_sq[i + 1] = h->off_sq[i] + ni * ni;
        h->off_I[i + 1] = h->off_I[i] + a;
        off_x[i + 1] = off_x[i] + ni * nt;
        off_m[i + 1] = off_m[i] + nt * nt;
        off_ti[i + 1] = off_ti[i] + (int64_t)a * 2 * a;
        off_P[i + 1] = off_P[i] + (int64_t)a * a;
        off_la[i + 1] = off_la[i] + (int64_t)cdiv(ni, CHOL_NB) * CHOL_NB * CHOL_NB;
        off_lm[i + 1] = off_lm[i] + (int64_t)cdiv(nR, CHOL_NB) * CHOL_NB * CHOL_NB;
        h->max_ni = std::max<int>(h->max_ni, (int)ni);
        h->max_nt = std::max<int>(h->max_nt, (int)nt);
    }
    h->sum_ni = h->off_om[N];
    h->sum_sq = h->off_sq[N];
    h->sum_nI = h->off_I[N];
    h->sum_nt = 0;
    for (int i = 0; i < N; ++i) {
        h->sum_nt += h->nt[i];
        h->apply_tri_elems += (int64_t)h->ni[i] * (h->ni[i] + 1);
    }

    // ---- gather plans for A_ii = R_i A R_i^T (order [I, G]) and for
    // X_i = R_i A tilde R_i^T with columns ordered [G, D, I] (Eq. (Xi)).
    std::vector<int32_t> omega(h->sum_ni);
    std::vector<int64_t> pa_src, pa_dst, px_src, px_dst;
    {
        std::vector<int32_t> stamp(n, -1), posA(n, -1), posX(n, -1);
        for (int i = 0; i < N; ++i) {
            const int nIi = h->nI[i], nGi = h->nG[i], ni = h->ni[i], nt = h->nt[i];
            const int nR = nGi + h->nD[i];
            int32_t* om = omega.data() + h->off_om[i];
            for (int a = 0; a < nIi; ++a) {
                const int32_t g = Il[i][a];
                om[a] = g;
                stamp[g] = i;
                posA[g] = a;
                posX[g] = nR + a;
            }
            for (int b = 0; b < nGi; ++b) {
                const int32_t g = Gl[i][b];
                om[nIi + b] = g;
                stamp[g] = i;
                posA[g] = nIi + b;
                posX[g] = b;
            }
            for (int c = 0; c < h->nD[i]; ++c) {
                const int32_t g = Dl[i][c];
                stamp[g] = i;
                posA[g] = -1;
                posX[g] = nGi + c;
            }
            for (int a = 0; a < ni; ++a) {
                const int32_t g = om[a];
                for (int64_t k = rp[g]; k < rp[g + 1]; ++k) {
                    const int32_t c = ci[k];
                    require(stamp[c] == i);  // every column of a row of Omega_i lies in tilde Omega_i
                    if (posA[c] >= 0) {
                        pa_src.push_back(k);
                        pa_dst.push_back(h->off_sq[i] + (int64_t)a * ni + posA[c]);
                    }
                    px_src.push_back(k);
                    px_dst.push_back(off_x[i] + (int64_t)a * nt + posX[c]);
                }
            }
        }
    }

    // ---- device buffers
    h->d_omega = C.up(omega, true);
    double* Araw = C.tnew<double>(h->sum_sq);
    T* Lb = C.tnew<T>(h->sum_sq);
    double* Xp = C.tnew<double>(off_x[N]);
    // the matrix-free eigensolve (eig_solver 3) forms none of Abar_ii, its
    // Schur complement or T_i
    const bool mf = h->eig_solver == 3;
    TS* M = C.tnew<TS>(mf ? 1 : off_m[N]);
    T* TI = C.tnew<T>(mf ? 1 : off_ti[N]);
    T* Pb = C.tnew<T>(mf ? 1 : off_P[N]);
    double* sig = C.tnew<double>(h->sum_ni);
    double* mu = C.tnew<double>(h->sum_nI);
    TS* delta = C.tnew<TS>(N);
    T* linvA = C.tnew<T>(off_la[N]);
    TS* linvM = C.tnew<TS>(mf ? 1 : off_lm[N]);
    // sweeps / rotations: [FP64 SVD, FP64 eig, FP32 SVD, FP32 eig] x N
    int* sweeps = C.tnew<int>(4 * N);
    unsigned long long* rots = C.tnew<unsigned long long>(4 * N);
    ck(cudaMemsetAsync(rots, 0, 4 * N * sizeof(unsigned long long), s));
    TS* nrmT = C.tnew<TS>(h->sum_ni);
    T* Yl = dnew<T>(h, h->sum_sq);   // L_i^{-1}
    T* Ylt = dnew<T>(h, h->sum_sq);  // L_i^{-T}
    if constexpr (f64) {
        h->d_Y = Yl;
        h->d_Yt = Ylt;
    } else {
        h->d_Y32 = Yl;
        h->d_Yt32 = Ylt;
    }
    ck(cudaMemsetAsync(Araw, 0, h->sum_sq * sizeof(double), s));
    ck(cudaMemsetAsync(Xp, 0, off_x[N] * sizeof(double), s));
    {
        const int64_t* sa = C.up(pa_src);
        const int64_t* da = C.up(pa_dst);
        const int64_t* sx = C.up(px_src);
        const int64_t* dx = C.up(px_dst);
        {
            PScope ps(h, PK_GATHER, 0.0, 32.0 * pa_src.size());
            launch_gather_values(sa, da, (int64_t)pa_src.size(), h->val, Araw, s);
        }
        {
            PScope ps(h, PK_GATHER, 0.0, 32.0 * px_src.size());
            launch_gather_values(sx, dx, (int64_t)px_src.size(), h->val, Xp, s);
        }
    }
    if constexpr (f64)
        ck(cudaMemcpyAsync(Lb, Araw, h->sum_sq * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else
        launch_convert<double, float>(Araw, Lb, h->sum_sq, s);

    // full selections: the basis diag(A_II)^{-1/2} keeps every block of E that
    // touches such a subdomain as sparse as A (its envelope-aware Cholesky and
    // the coarse solve then skip most tiles); with a kept E (multilevel form)
    // the A_II-orthonormal rows of L_A^{-1}, so that E is a block-orthogonal
    // congruence of the one any other A_II-orthonormal basis gives
    const bool diag_basis = !h->keep_E;
    h->diag_basis = diag_basis;
    // Z_i = diag(A_II)^{-1/2} for every fully selected subdomain (d_Zt allocated)
    auto fill_diag_zt = [&]() {
        std::vector<DiagBasisDesc> db;
        int maxn = 1;
        for (int i = 0; i < N; ++i)
            if (h->p[i] == h->nI[i] && h->p[i] > 0) {
                db.push_back({Araw + h->off_sq[i], h->ni[i], h->d_Zt + h->off_zt[i], h->nI[i]});
                maxn = std::max(maxn, h->nI[i]);
            }
        if (!db.empty()) {
            auto d = C.up(db);
            PScope ps(h, PK_SMALL);
            launch_diag_basis(d, (int)db.size(), maxn, h->s);
        }
    };
    // ---- (9) as a function of the selection (h->p, h->coff, h->d_Zt): the coarse
    // matrix, its ordering, factor and the diagonal-block inverses of the factor,
    // on whatever streams h->s / h->s2 name when it is called.
    auto factor_coarse = [&]() {
        // ---- (9) coarse matrix E = R_0 A R_0^T (Eq. (two_level_schwarz)), its
        // Cholesky factor and inverse factor
        cudaStream_t s = h->s;  // the stream this call runs on
        const int64_t nC = h->nC;
        h->d_cperm = nullptr;
        h->d_YEt = nullptr;
        h->d_cF = h->d_cG = nullptr;
        h->d_cfw0 = h->d_cgw1 = nullptr;
        h->cFW = 0;
        if (nC > 0) {
            std::vector<int64_t> off_az(N + 1, 0);
            for (int i = 0; i < N; ++i) off_az[i + 1] = off_az[i] + (int64_t)h->ni[i] * h->p[i];
            double* AZ = C.tnew<double>(off_az[N]);
            h->d_YE = dnew<double>(h, (size_t)nC * nC);  // E, then its Cholesky factor L_E (lower)
            double* E = h->d_YE;
            ck(cudaMemsetAsync(E, 0, (size_t)nC * nC * sizeof(double), s));
            std::vector<GemmDesc> g1, g2;
            std::vector<DiagScaleDesc> dsd;
            int max_ni_d = 1;
            for (int i = 0; i < N; ++i) {
                if (h->p[i] == 0) continue;
                const int ni = h->ni[i], nIi = h->nI[i], pi = h->p[i];
                if (diag_basis && pi == nIi) {
                    // Z_i = diag(A_II)^{-1/2}: AZ_i and E_ii are scalings of A_ii
                    // (the same products as the GEMMs, whose other terms are zeros)
                    dsd.push_back({Araw + h->off_sq[i], ni, nIi, AZ + off_az[i], E + (size_t)h->coff[i] * nC + h->coff[i],
                                   (int64_t)nC});
                    max_ni_d = std::max(max_ni_d, ni);
                    continue;
                }
                // AZ_i = A(Omega_i, Omega_Ii) Z_i   (ni x p_i)
                g1.push_back(gd(Araw + h->off_sq[i], ni, 0, h->d_Zt + h->off_zt[i], nIi, 1, AZ + off_az[i], pi, ni, pi,
                                nIi, 1.0, 0.0, 0));
                // E_ii = Z_i^T A_II Z_i
                g2.push_back(gd(h->d_Zt + h->off_zt[i], nIi, 0, AZ + off_az[i], pi, 0,
                                E + (size_t)h->coff[i] * nC + h->coff[i], (int)nC, pi, pi, nIi, 1.0, 0.0, 1));
            }
            gemm(C, g1);
            gemm(C, g2);
            if (!dsd.empty()) {
                auto d = C.up(dsd);
                PScope ps(h, PK_SMALL, 0.0, 0.0);
                launch_diag_scale(d, (int)dsd.size(), max_ni_d, s);
            }
            // E_ij (i > j) = sum over g in Omega_Ii cap Omega_j of Z_i[g]^T (A Z_j)[g]
            std::vector<int32_t> posI(n, -1);
            for (int i = 0; i < N; ++i)
                for (int a = 0; a < h->nI[i]; ++a) posI[Il[i][a]] = a;
            std::vector<std::vector<std::pair<int32_t, int32_t>>> lists;  // per pair
            std::vector<std::pair<int, int>> pairs;
            {
                std::vector<int> slot(N, -1);
                for (int j = 0; j < N; ++j) {
                    if (h->p[j] == 0) continue;
                    std::fill(slot.begin(), slot.end(), -1);
                    std::vector<int> touched;
                    const int32_t* om = omega.data() + h->off_om[j];
                    for (int ps = 0; ps < h->ni[j]; ++ps) {
                        const int32_t g = om[ps];
                        const int i = part[g];
                        if (i <= j || h->p[i] == 0) continue;
                        if (slot[i] < 0) {
                            slot[i] = (int)pairs.size();
                            pairs.push_back({i, j});
                            lists.emplace_back();
                        }
                        lists[slot[i]].push_back({posI[g], ps});
                    }
                }
            }
            std::vector<int32_t> la, lpos;
            std::vector<EPairRef> et;
            for (size_t q = 0; q < pairs.size(); ++q) {
                const int i = pairs[q].first, j = pairs[q].second;
                const int64_t lo = (int64_t)la.size();
                for (auto& e : lists[q]) {
                    la.push_back(e.first);
                    lpos.push_back(e.second);
                }
                for (int tr = 0; tr * 32 < h->p[i]; ++tr)
                    for (int tc = 0; tc * 32 < h->p[j]; ++tc) {
                        EPairRef t;
                        t.i = i;
                        t.j = j;
                        t.list_off = lo;
                        t.list_len = (int)lists[q].size();
                        t.tr = tr;
                        t.tc = tc;
                        et.push_back(t);
                    }
            }
            std::vector<int32_t> nIv(h->nI.begin(), h->nI.end()), pv(h->p.begin(), h->p.end());
            h->d_zt_off = C.up(std::vector<int64_t>(h->off_zt.begin(), h->off_zt.end() - 1), true);
            h->d_nI = C.up(nIv, true);
            h->d_p = C.up(pv, true);
            h->d_coff = C.up(std::vector<int64_t>(h->coff.begin(), h->coff.end() - 1), true);
            if (!et.empty()) {
                auto a = C.up(et);
                auto b = C.up(la);
                auto c = C.up(lpos);
                auto d = C.up(std::vector<int64_t>(off_az.begin(), off_az.end() - 1));
                double fl = 0.0;
                for (size_t q = 0; q < pairs.size(); ++q)
                    fl += 2.0 * h->p[pairs[q].first] * h->p[pairs[q].second] * lists[q].size();
                PScope ps(h, PK_E_ASM, fl);
                launch_e_offdiag(a, (int)et.size(), b, c, h->d_Zt, h->d_zt_off, h->d_nI, AZ, d, h->d_p, h->d_coff, E, nC,
                                 s);
            }
            if (h->keep_E) {
                // a copy of E for a next level (multilevel form), as a sparse matrix
                // with the block pattern: every entry of E_ij for i == j or for
                // subdomains coupled in A (a structural non-zero in
                // A(Omega_Ii, Omega_Ij)); E holds its lower triangle
                std::vector<std::vector<int>> adj(N);
                for (int64_t g = 0; g < n; ++g)
                    for (int64_t k = rp[g]; k < rp[g + 1]; ++k)
                        if (part[g] != part[ci[k]]) adj[part[g]].push_back(part[ci[k]]);
                for (int i = 0; i < N; ++i) {
                    adj[i].push_back(i);
                    std::sort(adj[i].begin(), adj[i].end());
                    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
                }
                std::vector<int64_t> erp(nC + 1, 0), esrc;
                std::vector<int32_t> ecol;
                for (int i = 0; i < N; ++i)
                    for (int k = 0; k < h->p[i]; ++k) {
                        const int64_t r = h->coff[i] + k;
                        for (int j : adj[i])
                            for (int l = 0; l < h->p[j]; ++l) {
                                const int64_t c = h->coff[j] + l;
                                ecol.push_back((int32_t)c);
                                esrc.push_back(std::max(r, c) * nC + std::min(r, c));
                            }
                        erp[r + 1] = (int64_t)ecol.size();
                    }
                h->E_nnz = (int64_t)ecol.size();
                h->d_E_rowptr = C.up(erp, true);
                h->d_E_col = C.up(ecol, true);
                h->d_E_val = dnew<double>(h, h->E_nnz);
                auto dsrc = C.up(esrc);
                PScope ps(h, PK_SMALL, 0.0, 16.0 * h->E_nnz);
                launch_gather_idx64(dsrc, h->E_nnz, E, h->d_E_val, s);
            }
            // ---- sparsity graph of E (coarse unknowns in subdomain order): blocks
            // of subdomains coupled in A (E_ij = Z_i^T A(Omega_Ii, Omega_Ij) Z_j is
            // exactly zero otherwise); a diagonal-basis block contributes only the
            // unknowns whose node touches the other subdomain
            std::vector<std::vector<int>> adjB(N);
            for (int64_t g = 0; g < n; ++g)
                for (int64_t q = rp[g]; q < rp[g + 1]; ++q)
                    if (part[g] != part[ci[q]]) adjB[part[g]].push_back(part[ci[q]]);
            for (int i = 0; i < N; ++i) {
                adjB[i].push_back(i);
                std::sort(adjB[i].begin(), adjB[i].end());
                adjB[i].erase(std::unique(adjB[i].begin(), adjB[i].end()), adjB[i].end());
            }
            auto full_diag = [&](int i) { return diag_basis && h->p[i] == h->nI[i] && h->p[i] > 0; };
            std::vector<std::vector<int32_t>> nbr(nC);
            for (int i = 0; i < N; ++i) {
                if (h->p[i] == 0) continue;
                if (full_diag(i)) {
                    for (int k = 0; k < h->p[i]; ++k) {
                        const int32_t g = Il[i][k];
                        auto& L = nbr[h->coff[i] + k];
                        for (int64_t q = rp[g]; q < rp[g + 1]; ++q) {
                            const int32_t g2 = ci[q];
                            const int j = part[g2];
                            if (h->p[j] == 0) continue;
                            if (full_diag(j))
                                L.push_back((int32_t)(h->coff[j] + posI[g2]));
                            else
                                for (int l = 0; l < h->p[j]; ++l) L.push_back((int32_t)(h->coff[j] + l));
                        }
                    }
                } else {
                    std::vector<int32_t> row;
                    for (int j : adjB[i]) {
                        if (h->p[j] == 0) continue;
                        if (!full_diag(j) || j == i) {
                            for (int l = 0; l < h->p[j]; ++l) row.push_back((int32_t)(h->coff[j] + l));
                        } else {
                            for (int l = 0; l < h->nI[j]; ++l) {  // nodes of Omega_Ij touching Omega_Ii
                                const int32_t g2 = Il[j][l];
                                for (int64_t q = rp[g2]; q < rp[g2 + 1]; ++q)
                                    if (part[ci[q]] == i) {
                                        row.push_back((int32_t)(h->coff[j] + l));
                                        break;
                                    }
                            }
                        }
                    }
                    for (int k = 0; k < h->p[i]; ++k) nbr[h->coff[i] + k] = row;
                }
            }
            for (auto& L : nbr) {
                std::sort(L.begin(), L.end());
                L.erase(std::unique(L.begin(), L.end()), L.end());
            }
            // ---- ordering of the coarse unknowns for the factorisation: reverse
            // Cuthill-McKee when it cuts the factorisation work (the sum over rows
            // of (r - first(r))^2) by a fifth or more, else the subdomain order.
            // E is permuted on the device; the coarse solves gather and scatter
            // through the order.
            auto envelope = [&](const std::vector<int32_t>& iperm, const std::vector<int32_t>& perm,
                                std::vector<int>& env) {
                env.assign(nC, 0);
                double work = 0.0;
                for (int64_t rn = 0; rn < nC; ++rn) {
                    int first = (int)rn;
                    for (int32_t c : nbr[perm[rn]]) first = std::min(first, (int)iperm[c]);
                    env[rn] = first;
                    work += (double)(rn - first) * (double)(rn - first);
                }
                return work;
            };
            std::vector<int32_t> idp(nC);
            std::iota(idp.begin(), idp.end(), 0);
            std::vector<int> env_id, env_rcm;
            const double prof_id = envelope(idp, idp, env_id);
            std::vector<int32_t> rperm = rcm_order(nbr);
            std::vector<int32_t> riperm(nC);
            for (int64_t q = 0; q < nC; ++q) riperm[rperm[q]] = (int32_t)q;
            const double prof_rcm = envelope(riperm, rperm, env_rcm);
            const bool use_rcm = prof_rcm < 0.8 * prof_id;
            h->env_row = use_rcm ? env_rcm : env_id;
            h->env_colend.assign(nC, 0);
            // the factor fills each row's envelope: column c of L_E reaches every
            // row whose envelope starts at or before c
            {
                std::vector<int> mark(nC, 0);
                for (int64_t r = 0; r < nC; ++r) mark[h->env_row[r]] = std::max(mark[h->env_row[r]], (int)r + 1);
                int run = 0;
                for (int64_t c = 0; c < nC; ++c) {
                    run = std::max(run, mark[c]);
                    h->env_colend[c] = std::max(run, (int)c + 1);
                }
            }
            double* linvE = C.tnew<double>((size_t)cdiv(nC, CHOL_NB) * CHOL_NB * CHOL_NB);
            if (use_rcm) {
                // E (lower triangle, subdomain order) -> Ep[r][c] = E[perm r][perm c]
                // (lower triangle); the two nC x nC buffers swap roles
                h->d_cperm = C.up(rperm, true);
                h->d_cp = dnew<double>(h, (size_t)MAXB * nC);
                h->d_ep = dnew<double>(h, (size_t)MAXB * nC);
                h->d_YEt = dnew<double>(h, (size_t)nC * nC);
                {
                    PScope ps(h, PK_SMALL, 0.0, 8.0 * (double)nC * nC);
                    launch_sym_permute(E, h->d_YEt, h->d_cperm, nC, s);
                }
                std::swap(h->d_YE, h->d_YEt);
                E = h->d_YE;
            }
            if (!h->d_YEt) h->d_YEt = dnew<double>(h, (size_t)nC * nC);
            chol_batched<double>(C, {CholDesc{E, (int)nC, (int)nC, (int)nC, nullptr, linvE}}, {&h->env_row});
            // Inverses of the diagonal blocks of L_E (block size cSB): the coarse
            // solve is then a blocked forward / backward substitution with L_E and
            // L_E^T, with no inverse of the whole factor.  About eight blocks, at
            // most 512 wide: each block costs two grid-wide phases per coarse
            // solve, and its inverse (stored dense) costs SB^3 / 3 FP64
            // multiply-adds in the setup, so n_C SB^2 / 3 in all.
            const int SB = std::min<int>(512, std::max<int>(CHOL_NB, cdiv(cdiv(nC, 8), CHOL_NB) * CHOL_NB));
            const int K = cdiv(nC, SB);
            h->cSB = SB;
            h->cK = K;
            h->d_Yd = dnew<double>(h, (size_t)K * SB * SB);
            h->d_Ydt = dnew<double>(h, (size_t)K * SB * SB);
            std::vector<TrtriDesc> tj;
            std::vector<const double*> ts;
            std::vector<double*> tdst;
            std::vector<int> tn, tl;
            for (int k = 0; k < K; ++k) {
                const int r0 = k * SB, sb = (int)std::min<int64_t>(SB, nC - r0);
                tj.push_back({E + (size_t)r0 * nC + r0, h->d_Yd + (size_t)k * SB * SB,
                              linvE + (size_t)(r0 / CHOL_NB) * CHOL_NB * CHOL_NB, sb, (int)nC, SB});
                ts.push_back(h->d_Yd + (size_t)k * SB * SB);
                tdst.push_back(h->d_Ydt + (size_t)k * SB * SB);
                tn.push_back(sb);
                tl.push_back(SB);
            }
            trtri_batched(C, tj);
            transpose_batched(C, ts, tdst, tn, tl, tl);
            transpose_batched<double>(C, {E}, {h->d_YEt}, {(int)nC}, {(int)nC}, {(int)nC});
            // folded coarse solve: when every block's rows reach back (and its
            // columns forward) at most SB entries beyond the block, F_k = Yd_k
            // L(block k, window) and G_k = Ydt_k L^T(block k, window) let each
            // block be solved in one grid-wide phase per direction
            {
                std::vector<int> fw0(K), gw1(K);
                int FW = 0;
                for (int k = 0; k < K; ++k) {
                    const int r0 = k * SB, r1 = (int)std::min<int64_t>(nC, (int64_t)r0 + SB);
                    int w0 = r0, w1 = r1;
                    for (int r = r0; r < r1; ++r) {
                        w0 = std::min(w0, h->env_row[r]);
                        w1 = std::max(w1, h->env_colend[r]);
                    }
                    fw0[k] = w0;
                    gw1[k] = w1;
                    FW = std::max(FW, std::max(r0 - w0, w1 - r1));
                }
                if (FW > 0 && FW <= SB) {
                    h->cFW = FW;
                    h->d_cF = dnew<double>(h, (size_t)K * SB * FW);
                    h->d_cG = dnew<double>(h, (size_t)K * SB * FW);
                    std::vector<GemmDesc> gfg;
                    for (int k = 0; k < K; ++k) {
                        const int r0 = k * SB, sb = (int)std::min<int64_t>(SB, nC - r0), r1 = r0 + sb;
                        const int W = r0 - fw0[k], V = gw1[k] - r1;
                        if (W > 0)
                            gfg.push_back(gd(h->d_Yd + (size_t)k * SB * SB, SB, 0, h->d_YE + (size_t)r0 * nC + fw0[k],
                                             (int)nC, 0, h->d_cF + (size_t)k * SB * FW, FW, sb, W, sb, 1.0, 0.0, 0));
                        if (V > 0)
                            gfg.push_back(gd(h->d_Ydt + (size_t)k * SB * SB, SB, 0, h->d_YEt + (size_t)r0 * nC + r1,
                                             (int)nC, 0, h->d_cG + (size_t)k * SB * FW, FW, sb, V, sb, 1.0, 0.0, 0));
                    }
                    gemm(C, gfg);
                    h->d_cfw0 = C.up(fw0, true);
                    h->d_cgw1 = C.up(gw1, true);
                }
            }
        } else {
            h->d_zt_off = C.up(std::vector<int64_t>(h->off_zt.begin(), h->off_zt.end() - 1), true);
            h->d_nI = C.up(std::vector<int32_t>(h->nI.begin(), h->nI.end()), true);
            h->d_p = C.up(std::vector<int32_t>(h->p.begin(), h->p.end()), true);
            h->d_coff = C.up(std::vector<int64_t>(h->coff.begin(), h->coff.end() - 1), true);
        }
    };

    // ---- speculative coarse space.  With Boolean D_i every non-zero eigenvalue
    // of eq. (Zi) is >= 1, so for tau > 1 every one is selected and the coarse
    // space is known before the eigensolve: the coarse matrix and its factor
    // (a latency-bound FP64 chain on few SMs) are built on the third and fourth
    // streams while the local eigenproblems run.  The selection computed in
    // step (7) is then compared with this one; on a mismatch (rounding below
    // 1/tau) the speculative work is dropped and step (9) runs as usual.
    const bool spec = diag_basis && h->tau >= 1.01 && h->s3 && h->s4;
    bool spec_ok = false;
    std::vector<int32_t> spec_p;
    if (spec) {
        h->p.assign(h->nI.begin(), h->nI.end());
        h->coff.assign(N + 1, 0);
        h->off_zt.assign(N + 1, 0);
        for (int i = 0; i < N; ++i) {
            h->coff[i + 1] = h->coff[i] + h->p[i];
            h->off_zt[i + 1] = h->off_zt[i] + (int64_t)h->p[i] * h->nI[i];
        }
        h->nC = h->coff[N];
        h->sum_zt = h->off_zt[N];
        spec_p = h->p;
        ck(cudaEventRecord(h->ev_spec_in, h->s));  // A_ii gathered
        ck(cudaStreamWaitEvent(h->s3, h->ev_spec_in, 0));
        std::swap(h->s, h->s3);
        std::swap(h->s2, h->s4);
        std::swap(h->ev_panel, h->ev_panel3);
        std::swap(h->ev_far, h->ev_far3);
        auto restore = [&]() {
            std::swap(h->s, h->s3);
            std::swap(h->s2, h->s4);
            std::swap(h->ev_panel, h->ev_panel3);
            std::swap(h->ev_far, h->ev_far3);
        };
        try {
            h->d_Zt = dnew<double>(h, h->sum_zt);
            fill_diag_zt();
            factor_coarse();
            ck(cudaEventRecord(h->ev_spec_done, h->s));
        } catch (...) {
            restore();
            throw;
        }
        restore();
    }

    // ---- (1) exact Cholesky of A_ii (local solver) and its inverse factor
    {
        std::vector<CholDescT<T>> cd(N);
        std::vector<TrtriDescT<T>> td(N);
        std::vector<const T*> src(N);
        std::vector<T*> dst(N);
        std::vector<int> nn(N), ld(N);
        for (int i = 0; i < N; ++i) {
            const int ni = h->ni[i];
            cd[i] = {Lb + h->off_sq[i], ni, ni, ni, nullptr, linvA + off_la[i]};
            td[i] = {Lb + h->off_sq[i], Yl + h->off_sq[i], linvA + off_la[i], ni, ni, ni};
            src[i] = Yl + h->off_sq[i];
            dst[i] = Ylt + h->off_sq[i];
            nn[i] = ni;
            ld[i] = ni;
        }
        chol_batched(C, cd);
        trtri_batched(C, td);
        transpose_batched(C, src, dst, nn, ld, ld);
    }

    // ---- (1b) sparse Cholesky factors of the A_ii in a nested-dissection order
    // (Sec. 4.1: exact local Cholesky; the same factor of the permuted matrix,
    // with the fill of the symbolic factorisation only): local solves then read
    // the factor's entries instead of the dense triangles of L_i^{-1}.
    if (h->local_solver != 0) build_sparse_local<T>(C, h, rp, ci, omega);

    // ---- (2) SVD of X_i (Sec. 3.2) by one-sided Jacobi on its rows: an
    // FP32-preconditioned rotation Q_i (orthogonal to FP64 accuracy) is applied
    // in FP64, X1_i = Q_i X_i, then FP64 sweeps make the rows of X1_i exactly
    // orthogonal: rows become sigma_j v_j^T, sigma_j = row norms; rows are then
    // scaled by sigma_j^{-1/2}.
    // eps is the machine precision of the arithmetic (Sec. 3.2): the FP32
    // stage shifts by at least sigma_1 * 2^-23, above its own rounding.
    if constexpr (!s64) h->eps = std::max(h->eps, (double)std::numeric_limits<float>::epsilon());
    const double eps = h->eps;
    TS* X1 = C.tnew<TS>(off_x[N]);
    if constexpr (s64) {
        std::vector<int64_t> oq(N + 1, 0);
        for (int i = 0; i < N; ++i) oq[i + 1] = oq[i] + (int64_t)h->ni[i] * h->ni[i];
        double* Q = C.tnew<double>(oq[N]);
        std::vector<PrecondJob> pj(N);
        std::vector<GemmDesc> g(N);
        for (int i = 0; i < N; ++i) {
            pj[i] = {Xp + off_x[i], h->ni[i], h->nt[i], h->nt[i], Q + oq[i]};
            g[i] = gd(Q + oq[i], h->ni[i], 0, Xp + off_x[i], h->nt[i], 0, X1 + off_x[i], h->nt[i], h->ni[i],
                      h->nt[i], h->ni[i], 1.0, 0.0, 0);
        }
        fp32_precondition(C, pj, false, 40, sweeps + 2 * N, rots + 2 * N);
        gemm(C, g);
        std::vector<JacobiDesc> jd(N);
        std::vector<double*> sp(N);
        int maxc = 1;
        for (int i = 0; i < N; ++i) {
            jd[i] = {X1 + off_x[i], h->ni[i], h->nt[i], h->nt[i], h->nt[i], nrmT + h->off_om[i], nullptr};
            sp[i] = sig + h->off_om[i];
            maxc = std::max(maxc, h->nt[i]);
        }
        JacobiDesc* djd = C.up(jd);
        double* const* dsp = C.up(sp);
        {
            PScope ps(h, PK_JAC_SVD);
            run_jacobi<double>(C, jd, djd, h->max_sweeps,
                               2.0 * std::sqrt((double)maxc) * std::numeric_limits<double>::epsilon(), sweeps, rots, 1);
        }
        PScope ps(h, PK_SMALL);
        launch_rownorms(djd, N, dsp, delta, eps, 1, s);
    }

    else {
        // FP32 splitting: one-sided Jacobi on the rows of X_i alone
        launch_convert<double, float>(Xp, X1, off_x[N], s);
        std::vector<JacobiDescT<float>> jd(N);
        std::vector<double*> sp(N);
        int maxc = 1;
        for (int i = 0; i < N; ++i) {
            jd[i] = {X1 + off_x[i], h->ni[i], h->nt[i], h->nt[i], h->nt[i], nrmT + h->off_om[i], nullptr};
            sp[i] = sig + h->off_om[i];
            maxc = std::max(maxc, h->nt[i]);
        }
        JacobiDescT<float>* djd = C.up(jd);
        double* const* dsp = C.up(sp);
        {
            PScope ps(h, PK_JAC_F32);
            run_jacobi<float>(C, jd, djd, h->max_sweeps,
                              8.0f * std::sqrt((float)maxc) * std::numeric_limits<float>::epsilon(), sweeps, rots, 0);
        }
        PScope ps(h, PK_SMALL);
        launch_rownorms<float>(djd, N, dsp, delta, eps, 1, s);
    }

    // steps (3)-(6): the splitting, its Schur complement, T_i and its eigenvalues
    if (!mf) {
        // ---- (3) Abar_ii = C^T diag(1/sigma) C + sigma_1 eps I, ordered [G, D, I]
        {
            std::vector<GemmDescT<TS>> g(N);
            std::vector<TS*> mats(N);
            std::vector<int> nn(N), ld(N);
            for (int i = 0; i < N; ++i) {
                const int ni = h->ni[i], nt = h->nt[i];
                TS* Xi = X1 + off_x[i];
                g[i] = gd(Xi, nt, 1, Xi, nt, 0, M + off_m[i], nt, nt, nt, ni, 1.0, 0.0, 1);
                mats[i] = M + off_m[i];
                nn[i] = nt;
                ld[i] = nt;
            }
            gemm(C, g);
            auto a = C.up(mats);
            auto b = C.up(nn);
            auto c = C.up(ld);
            PScope ps(h, PK_SMALL);
            launch_add_diag<TS>(a, b, c, delta, N, h->max_nt, s);
        }

        // ---- (4) Schur complement of Abar_ii onto Omega_Ii: Cholesky of the
        // leading [G, D] block (pivot floor sigma_1 eps, the shift of Remark 3.2).
        constexpr bool f64s = std::is_same<TS, double>::value;
        int* dbad = C.tnew<int>(N);
        ck(cudaMemsetAsync(dbad, 0, N * sizeof(int), s));
        {
            std::vector<CholDescT<TS>> cd(N);
            for (int i = 0; i < N; ++i) {
                const int nt = h->nt[i], nR = h->nG[i] + h->nD[i];
                cd[i] = {M + off_m[i], nt, nt, nR, delta + i, linvM + off_lm[i], dbad + i};
            }
            chol_batched(C, cd);
        }

        // ---- (5) T = L_A^{-1} S L_A^{-T} (L_A = Cholesky factor of A_II, the
        // leading block of that of A_ii), appended identity for the rotations.
        // With an FP64 splitting and FP32 local work, S is rounded to FP32 first.
        {
            std::vector<TS*> mats(N);
            std::vector<int> nn(N), ld(N);
            std::vector<GemmDescT<T>> g1(N), g2(N);
            std::vector<TrtriDescT<T>> idd(N);
            T* Sc = nullptr;
            if constexpr (!std::is_same<T, TS>::value) Sc = C.tnew<T>(off_P[N]);
            std::vector<const TS*> csrc(N);
            std::vector<T*> cdst(N);
            std::vector<int> cls(N), cld(N);
            for (int i = 0; i < N; ++i) {
                const int nIi = h->nI[i], nt = h->nt[i], nR = h->nG[i] + h->nD[i], ni = h->ni[i];
                TS* S = M + off_m[i] + (size_t)nR * nt + nR;
                mats[i] = S;
                nn[i] = nIi;
                ld[i] = nt;
                const T* Y = Yl + h->off_sq[i];
                const T* Sl;
                int lds;
                if constexpr (std::is_same<T, TS>::value) {
                    Sl = S;
                    lds = nt;
                } else {
                    Sl = Sc + off_P[i];
                    lds = nIi;
                }
                csrc[i] = S;
                cdst[i] = Sc ? Sc + off_P[i] : nullptr;
                cls[i] = nt;
                cld[i] = nIi;
                g1[i] = gd(Y, ni, 0, Sl, lds, 0, Pb + off_P[i], nIi, nIi, nIi, nIi, 1.0, 0.0, 0);
                g2[i] = gd(Pb + off_P[i], nIi, 0, Y, ni, 1, TI + off_ti[i], 2 * nIi, nIi, nIi, nIi, 1.0, 0.0, 0);
                idd[i] = {nullptr, TI + off_ti[i] + nIi, nullptr, nIi, 0, 2 * nIi};
            }
            {
                auto a = C.up(mats);
                auto b = C.up(nn);
                auto c = C.up(ld);
                PScope ps(h, PK_SMALL);
                launch_mirror_lower<TS>(a, b, c, N, h->max_nt, s);
            }
            if constexpr (!std::is_same<T, TS>::value) {
                auto a = C.up(csrc);
                auto b = C.up(cls);
                auto c = C.up(cdst);
                auto d = C.up(cld);
                auto e = C.up(nn);
                PScope ps(h, PK_SMALL);
                launch_convert_blocks<TS, T>(a, b, c, d, e, N, h->max_nt, s);
            }
            gemm(C, g1);
            gemm(C, g2);
            auto di = C.up(idd);
            PScope ps(h, PK_SMALL);
            launch_set_identity<T>(di, N, h->max_nt, s);
        }

        // ---- (5b) robust Schur complement for the subdomains whose clamped
        // Cholesky was flagged.  With C = Sigma^{1/2} V^T = [C_R | C_I] (the scaled
        // rows of step (2), columns [G, D | I]) and Abar = C^T C + delta I, the
        // push-through identity gives the Schur complement onto Omega_Ii as
        //   S = delta (I + C_I^T (C_R C_R^T + delta I)^{-1} C_I).
        // C_R C_R^T + delta I = Q^T diag(s_k^2 + delta) Q comes from a one-sided
        // Jacobi of the rows of C_R (no Gram matrix is formed, so the shift is
        // never swamped by rounding), W = diag(1 / sqrt(s^2 + delta)) Q C_I and
        //   T = L_A^{-1} S L_A^{-T} = delta (L_A^{-1} L_A^{-T} + P^T P),  P = W L_A^{-T},
        // a sum of positive semidefinite terms.
        {
            std::vector<int> bad(N);
            std::vector<TS> dl(N);
            ck(cudaMemcpyAsync(bad.data(), dbad, N * sizeof(int), cudaMemcpyDeviceToHost, s));
            ck(cudaMemcpyAsync(dl.data(), delta, N * sizeof(TS), cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            std::vector<int> F;
            for (int i = 0; i < N; ++i)
                if (bad[i] && h->nG[i] + h->nD[i] > 0) F.push_back(i);
            h->n_robust = (int)F.size();
            if (!F.empty()) {
                const int nf = (int)F.size();
                std::vector<int64_t> oj(nf + 1, 0), ow(nf + 1, 0);
                for (int q = 0; q < nf; ++q) {
                    const int i = F[q];
                    oj[q + 1] = oj[q] + (int64_t)h->ni[i] * (h->nG[i] + h->nD[i] + h->ni[i]);
                    ow[q + 1] = ow[q] + (int64_t)h->ni[i] * h->nI[i];
                }
                TS* J = C.tnew<TS>(oj[nf]);
                TS* W = C.tnew<TS>(ow[nf]);
                TS* nrm = C.tnew<TS>(h->sum_ni);
                std::vector<KjacDesc<TS>> kd(nf);
                std::vector<JacobiDescT<TS>> jd(nf);
                int maxr = 1, maxc = 1;
                for (int q = 0; q < nf; ++q) {
                    const int i = F[q], ni = h->ni[i], nt = h->nt[i], nR = h->nG[i] + h->nD[i], lj = nR + ni;
                    kd[q] = {X1 + off_x[i], J + oj[q], ni, nR, nt, lj, delta + i};
                    jd[q] = {J + oj[q], ni, lj, nR, lj, nrm + h->off_om[i], nullptr};
                    maxr = std::max(maxr, ni);
                    maxc = std::max(maxc, nR);
                }
                // no rotation for |<p,q>| <= tol * delta: such rows are resolved to
                // the accuracy of K = C_R C_R^T + delta I already
                std::vector<TS> kfl(nf);
                const TS tol = (f64s ? TS(2) : TS(8)) * std::sqrt((TS)maxc) * std::numeric_limits<TS>::epsilon();
                for (int q = 0; q < nf; ++q) kfl[q] = tol * dl[F[q]];
                TS* dkfl = C.up(kfl);
                for (int q = 0; q < nf; ++q) jd[q].absfloor = dkfl + q;
                auto dkd = C.up(kd);
                JacobiDescT<TS>* djd = C.up(jd);
                int* rsw = C.tnew<int>(nf);
                unsigned long long* rrot = C.tnew<unsigned long long>(nf);
                {
                    PScope ps(h, PK_SMALL);
                    launch_build_kjac<TS>(dkd, nf, maxr, s);
                }
                {
                    PScope ps(h, pk<TS>(PK_JAC_SVD, PK_JAC_F32));
                    run_jacobi<TS>(C, jd, djd, h->max_sweeps, tol, rsw, rrot, f64s ? 1 : 0);
                }
                {
                    PScope ps(h, PK_SMALL);
                    launch_kjac_scale<TS>(dkd, nf, s);
                }
                std::vector<GemmDescT<TS>> gw(nf);
                for (int q = 0; q < nf; ++q) {
                    const int i = F[q], ni = h->ni[i], nt = h->nt[i], nR = h->nG[i] + h->nD[i], nIi = h->nI[i];
                    gw[q] = gd<TS>(J + oj[q] + nR, nR + ni, 0, X1 + off_x[i] + nR, nt, 0, W + ow[q], nIi, ni, nIi, ni,
                                   1.0, 0.0, 0);
                }
                gemm(C, gw);
                T* WT = nullptr;
                if constexpr (std::is_same<T, TS>::value) {
                    WT = W;
                } else {
                    WT = C.tnew<T>(ow[nf]);
                    launch_convert<TS, T>(W, WT, ow[nf], s);
                }
                T* P = C.tnew<T>(ow[nf]);
                std::vector<GemmDescT<T>> g1, g2;
                for (int q = 0; q < nf; ++q) {
                    const int i = F[q], ni = h->ni[i], nIi = h->nI[i];
                    const T* Y = Yl + h->off_sq[i];  // L_A^{-1}: leading nI x nI block of L_i^{-1}
                    const double dv = (double)dl[i];
                    g1.push_back(gd<T>(WT + ow[q], nIi, 0, Y, ni, 1, P + ow[q], nIi, ni, nIi, nIi, 1.0, 0.0, 0));
                    g1.push_back(gd<T>(Y, ni, 0, Y, ni, 1, TI + off_ti[i], 2 * nIi, nIi, nIi, nIi, dv, 0.0, 0));
                    g2.push_back(gd<T>(P + ow[q], nIi, 1, P + ow[q], nIi, 0, TI + off_ti[i], 2 * nIi, nIi, nIi, ni, dv,
                                       1.0, 0));
                }
                gemm(C, g1);
                gemm(C, g2);
            }
        }

        // ---- (6) eigenvalues mu = 1/lambda of eq. (Zi): Householder reduction of
        // each T_i to tridiagonal form and bisection with Sturm counts (absolute
        // accuracy O(eps ||T||), like a dense symmetric eigensolver).
        {
            T* TD = C.tnew<T>(off_P[N]);
            T* dd = C.tnew<T>(h->sum_nI);
            T* ee = C.tnew<T>(h->sum_nI);
            T* pp = C.tnew<T>(h->sum_nI);
            std::vector<TridiagDescT<T>> td(N);
            std::vector<double*> outp(N);
            std::vector<int> em, ej;
            em.reserve(h->sum_nI);
            ej.reserve(h->sum_nI);
            int maxn = 1;
            for (int i = 0; i < N; ++i) {
                const int nIi = h->nI[i];
                if (nIi > 0)
                    ck(cudaMemcpy2DAsync(TD + off_P[i], nIi * sizeof(T), TI + off_ti[i], 2 * nIi * sizeof(T),
                                         nIi * sizeof(T), nIi, cudaMemcpyDeviceToDevice, s));
                td[i] = {TD + off_P[i], nIi, nIi, dd + h->off_I[i], ee + h->off_I[i], pp + h->off_I[i]};
                outp[i] = mu + h->off_I[i];
                for (int j = 0; j < nIi; ++j) {
                    em.push_back(i);
                    ej.push_back(j);
                }
                maxn = std::max(maxn, nIi);
            }
            const TridiagDescT<T>* dtd = C.up(td);
            auto dem = C.up(em);
            auto dej = C.up(ej);
            auto dout = C.up(outp);
            {
                double fl = 0.0;
                for (int i = 0; i < N; ++i) fl += 8.0 / 3.0 * std::pow((double)h->nI[i], 3);
                PScope ps(h, pk<T>(PK_TRIDIAG, PK_TRIDIAG_F32), fl);
                launch_tridiag<T>(dtd, N, maxn, s);
            }
            PScope ps(h, pk<T>(PK_BISECT, PK_BISECT_F32));
            launch_bisect<T>(dtd, N, dem, dej, (int64_t)em.size(), dout, s);
        }
    }  // !mf

    // ---- (6mf) the matrix-free eigensolve of eq. (Zi) through eq. (invAii)
    std::vector<std::vector<double>> mf_lam;
    std::vector<double*> mf_rows;
    std::vector<int> mf_its;
    if constexpr (f64 && s64) {
        if (mf) mf_local_eigs(C, h, X1, off_x, sig, delta, Lb, mf_lam, mf_rows, mf_its);
    }

    // ---- (7) selection lambda > 1/tau on the host
    std::vector<double> mu_h(h->sum_nI);
    std::vector<int> sw(4 * N);
    std::vector<unsigned long long> rot_h(4 * N);
    h->sigma_h.resize(h->sum_ni);
    ck(cudaMemcpyAsync(rot_h.data(), rots, 4 * N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    if (!mf) ck(cudaMemcpyAsync(mu_h.data(), mu, h->sum_nI * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(h->sigma_h.data(), sig, h->sum_ni * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(sw.data(), sweeps, 4 * N * sizeof(int), cudaMemcpyDeviceToHost, s));
    {
        const int e = read_err(h);
        if (e) throw Fail{err_status(e)};
    }
    for (int i = 0; i < N; ++i) {
        h->sweeps_svd = std::max(h->sweeps_svd, sw[i]);
        h->sweeps_svd32 = std::max(h->sweeps_svd32, sw[2 * N + i]);
        h->rot_svd += (int64_t)rot_h[i];
        if (h->prof.on) {
            // per sweep: row norms and one inner product per pair; plus the rotations performed
            const double ni = h->ni[i], nt = h->nt[i];
            // (the class of the precision the SVD ran in)
            h->prof.flops[pk<TS>(PK_JAC_SVD, PK_JAC_F32)] +=
                sw[i] * (ni * 2.0 * nt + ni * (ni - 1) / 2 * 2.0 * nt) + rot_h[i] * 6.0 * nt;
        }
        std::sort(h->sigma_h.begin() + h->off_om[i], h->sigma_h.begin() + h->off_om[i + 1], std::greater<double>());
    }
    h->lam_h.resize(h->sum_nI);
    h->p.assign(N, 0);
    h->coff.assign(N + 1, 0);
    h->off_zt.assign(N + 1, 0);
    std::vector<int> partial;  // subdomains whose selection is neither empty nor everything
    for (int i = 0; i < N; ++i) {
        const int nIi = h->nI[i];
        int pi = 0;
        for (int j = 0; j < nIi; ++j) {  // mu ascending -> lambda descending
            double lam;
            if (mf) {  // the computed ones (descending), NaN for the rest
                lam = j < (int)mf_lam[i].size() ? mf_lam[i][j] : std::numeric_limits<double>::quiet_NaN();
            } else {
                const double m = mu_h[h->off_I[i] + j];
                lam = (m > 0.0) ? 1.0 / m : std::numeric_limits<double>::infinity();
            }
            h->lam_h[h->off_I[i] + j] = lam;
            if (lam > 1.0 / h->tau) ++pi;
            // below 1: possible only through the shift sigma_1 eps of the splitting
            // (diagnostic count)
            if (lam < 1.0 - 1e-6) ++h->n_below_one;
            if (std::fabs(lam * h->tau - 1.0) <= h->tie_band) ++h->n_tied;
        }
        h->p[i] = pi;
        if (pi > 0 && pi < nIi) partial.push_back(i);
        h->coff[i + 1] = h->coff[i] + pi;
        h->off_zt[i + 1] = h->off_zt[i] + (int64_t)pi * nIi;
    }
    h->nC = h->coff[N];
    h->sum_zt = h->off_zt[N];
    if (spec) {
        spec_ok = h->p == spec_p;
        if (spec_ok) {
            ck(cudaStreamWaitEvent(s, h->ev_spec_done, 0));
        } else {  // the speculative buffers stay owned by the handle until amdd_destroy
            ck(cudaStreamSynchronize(h->s3));
            ck(cudaStreamSynchronize(h->s4));
        }
    }

    // ---- (8) coarse block Z_i on Omega_Ii as A_II-orthonormal rows.  When
    // every eigenvalue is selected, span(Z_i) = R^{|Omega_Ii|} and any
    // A_II-orthonormal basis serves: the rows of L_A^{-1}.  When the selection
    // is partial, the eigenvectors are needed: one-sided Jacobi on the rows of
    // [T | I] (FP64, relative criterion) gives the eigenvectors w_j as the
    // right half and mu_j as the left-half row norms; the p_i rows with the
    // smallest mu give u = L_A^{-T} w.
    if (spec_ok) {
        h->n_partial = 0;
        h->eig_iters.assign(N, -2);
        if (mf) h->eig_iters = mf_its;
    } else {
        h->d_Zt = dnew<double>(h, h->sum_zt);
        T* ZtT = nullptr;
        if constexpr (f64)
            ZtT = h->d_Zt;
        else
            ZtT = C.tnew<T>(h->sum_zt);
        // full selections: the basis diag(A_II)^{-1/2} keeps every block of E that
        // touches such a subdomain as sparse as A (its envelope-aware Cholesky and
        // the coarse solve then skip most tiles); with a kept E (multilevel form)
        // the A_II-orthonormal rows of L_A^{-1}, so that E is a block-orthogonal
        // congruence of the one any other A_II-orthonormal basis gives
        if (h->nC > 0) {
            std::vector<int64_t> ysrc, ydst;
            std::vector<int32_t> ylen;
            for (int i = 0; i < N; ++i) {
                if (h->p[i] != h->nI[i] || h->p[i] == 0 || diag_basis) continue;
                for (int k = 0; k < h->nI[i]; ++k) {
                    ysrc.push_back(h->off_sq[i] + (int64_t)k * h->ni[i]);
                    ydst.push_back(h->off_zt[i] + (int64_t)k * h->nI[i]);
                    ylen.push_back(h->nI[i]);
                }
            }
            if (!ysrc.empty()) {
                auto a = C.up(ysrc);
                auto b = C.up(ydst);
                auto c = C.up(ylen);
                PScope ps(h, PK_SMALL);
                launch_gather_rows<T>(Yl, a, ZtT, b, c, (int64_t)ysrc.size(), s);
            }
            h->n_partial = (int)partial.size();
            h->eig_iters.assign(N, -2);
            if (mf) h->eig_iters = mf_its;
            T* Wsel = partial.empty() ? nullptr : C.tnew<T>(h->sum_zt);
            std::vector<int> dense = partial;  // subdomains whose eigenvectors come from the dense Jacobi
            if (mf) {
                // the leading p_i Ritz rows of the matrix-free eigensolve
                // (descending lambda, contiguous p_i x nI blocks)
                if constexpr (f64)
                    for (int i : partial)
                        ck(cudaMemcpyAsync(Wsel + h->off_zt[i], mf_rows[i], (size_t)h->p[i] * h->nI[i] * sizeof(T),
                                           cudaMemcpyDeviceToDevice, s));
                dense.clear();
            } else if (!partial.empty() && (h->eig_solver >= 1 || h->keep_prop)) {
                dense = learned_eigvecs<T>(C, h, partial, Araw, Lb, TI, off_ti, Wsel);
            }
            for (int i : dense) h->eig_iters[i] = -1;
            if (!dense.empty()) {
                const std::vector<int>& partial_d = dense;
                const int np = (int)partial_d.size();
                std::vector<JacobiDescT<T>> jd(np);
                std::vector<double*> mp(np);
                double* mu_j = C.tnew<double>(h->sum_nI);
                T* nrmE = C.tnew<T>(h->sum_nI);  // row norms of the eigen-Jacobi
                int maxc = 1;
                for (int q = 0; q < np; ++q) {
                    const int i = partial_d[q], nIi = h->nI[i];
                    jd[q] = {TI + off_ti[i], nIi, 2 * nIi, nIi, 2 * nIi, nrmE + h->off_I[i], nullptr};
                    mp[q] = mu_j + h->off_I[i];
                    maxc = std::max(maxc, nIi);
                }
                JacobiDescT<T>* djd = C.up(jd);
                double* const* dmp = C.up(mp);
                {
                    PScope ps(h, PK_JAC_EIG);
                    const T tol = (f64 ? T(2) : T(8)) * std::sqrt((T)maxc) * std::numeric_limits<T>::epsilon();
                    run_jacobi<T>(C, jd, djd, h->max_sweeps, tol, sweeps + N, rots + N, f64 ? 1 : 0);
                }
                {
                    PScope ps(h, PK_SMALL);
                    launch_rownorms<T>(djd, np, dmp, (T*)nullptr, 0.0, 0, s);
                }
                std::vector<double> muj(h->sum_nI);
                ck(cudaMemcpyAsync(muj.data(), mu_j, h->sum_nI * sizeof(double), cudaMemcpyDeviceToHost, s));
                ck(cudaMemcpyAsync(sw.data() + N, sweeps + N, N * sizeof(int), cudaMemcpyDeviceToHost, s));
                ck(cudaMemcpyAsync(rot_h.data() + N, rots + N, N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
                {
                    const int e = read_err(h);
                    if (e) throw Fail{err_status(e)};
                }
                std::vector<int64_t> wsrc, wdst;
                std::vector<int32_t> wlen;
                for (int q = 0; q < np; ++q) {
                    const int i = partial_d[q], nIi = h->nI[i];
                    h->sweeps_eig = std::max(h->sweeps_eig, sw[N + q]);
                    h->rot_eig += (int64_t)rot_h[N + q];
                    if (h->prof.on)
                        h->prof.flops[PK_JAC_EIG] +=
                            sw[N + q] * (nIi * 2.0 * nIi + nIi * (nIi - 1) / 2.0 * 2.0 * nIi) + rot_h[N + q] * 12.0 * nIi;
                    std::vector<int> order(nIi);
                    std::iota(order.begin(), order.end(), 0);
                    const double* m = muj.data() + h->off_I[i];
                    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return m[x] < m[y]; });
                    for (int k = 0; k < h->p[i]; ++k) {
                        wsrc.push_back(off_ti[i] + (int64_t)order[k] * 2 * nIi + nIi);
                        wdst.push_back(h->off_zt[i] + (int64_t)k * nIi);
                        wlen.push_back(nIi);
                    }
                }
                {
                    auto a = C.up(wsrc);
                    auto b = C.up(wdst);
                    auto c = C.up(wlen);
                    PScope ps(h, PK_SMALL);
                    launch_gather_rows<T>(TI, a, Wsel, b, c, (int64_t)wsrc.size(), s);
                }
            }
            if (!partial.empty()) {
                std::vector<GemmDescT<T>> g;
                for (int i : partial)
                    g.push_back(gd<T>(Wsel + h->off_zt[i], h->nI[i], 0, Yl + h->off_sq[i], h->ni[i], 0,
                                      ZtT + h->off_zt[i], h->nI[i], h->p[i], h->nI[i], h->nI[i], 1.0, 0.0, 0));
                gemm(C, g);
            }
            // the coarse part is FP64: Z_i rounded to FP64 once, used for E and the apply
            if constexpr (!f64) launch_convert<float, double>(ZtT, h->d_Zt, h->sum_zt, s);
            if (diag_basis) fill_diag_zt();
        }
        if (mf) h->eig_iters = mf_its;
    }

    if (!spec_ok) factor_coarse();
    const int64_t nC = h->nC;

    // ---- (10) apply plan
    {
        std::vector<GemvDescT<T>> l1(N), l2(N);
        std::vector<GemvDesc> cr(N);
        h->d_rloc = dnew<double>(h, h->sum_ni);
        T* rlocT = f64 ? (T*)h->d_rloc : dnew<T>(h, h->sum_ni);
        T* tlocT = dnew<T>(h, h->sum_ni);
        T* ylocT = dnew<T>(h, h->sum_ni);
        if constexpr (f64) {
            h->d_tloc = tlocT;
            h->d_yloc = ylocT;
        } else {
            h->d_rloc32 = rlocT;
            h->d_tloc32 = tlocT;
            h->d_yloc32 = ylocT;
        }
        h->d_c = dnew<double>(h, nC);
        h->d_e = dnew<double>(h, nC);
        if (nC > 0) {
            h->d_Zr = dnew<double>(h, h->sum_zt);
            h->d_zc = dnew<double>(h, n);
            ck(cudaMemsetAsync(h->d_zc, 0, n * sizeof(double), s));
            std::vector<TransDesc> tdz;
            std::vector<int32_t> rdz, rlz;
            int maxd = 1;
            h->gv_zp_h.clear();
            for (int i = 0; i < N; ++i) {
                if (h->p[i] == 0) continue;
                const int pi = h->p[i], nIi = h->nI[i];
                tdz.push_back({h->d_Zt + h->off_zt[i], h->d_Zr + h->off_zt[i], pi, nIi, nIi, pi});
                maxd = std::max(maxd, std::max(pi, nIi));
                GemvDesc g{h->d_Zr + h->off_zt[i], nIi, pi, pi, 0, h->d_e + h->coff[i], h->d_zc + h->off_I[i]};
                for (int a = 0; a < nIi; ++a) {
                    rdz.push_back((int32_t)h->gv_zp_h.size());
                    rlz.push_back(a);
                }
                h->gv_zp_h.push_back(g);
            }
            auto dt = C.up(tdz);
            {
                PScope ps(h, PK_SMALL);
                launch_transpose_rect(dt, (int)tdz.size(), maxd, s);
            }
            h->d_gv_zp = C.up(h->gv_zp_h, true);
            h->d_rd_zp = C.up(rdz, true);
            h->d_rl_zp = C.up(rlz, true);
            h->n_zp = (int64_t)rdz.size();
        }
        std::vector<int32_t> rd, rl, rdc, rlc;  // rd / rl: row groups of the local products (matrix, first row)
        h->lm1.assign(N, nullptr);
        h->lm2.assign(N, nullptr);
        for (int i = 0; i < N; ++i) {
            const int ni = h->ni[i];
            h->lm1[i] = Yl + h->off_sq[i];
            h->lm2[i] = Ylt + h->off_sq[i];
            l1[i] = {Yl + h->off_sq[i], ni, ni, ni, 1, rlocT + h->off_om[i], tlocT + h->off_om[i]};
            l2[i] = {Ylt + h->off_sq[i], ni, ni, ni, 2, tlocT + h->off_om[i], ylocT + h->off_om[i]};
            cr[i] = {h->d_Zt + h->off_zt[i], h->p[i], h->nI[i], h->nI[i], 0, h->d_rloc + h->off_om[i],
                     h->d_c + h->coff[i]};
            for (int a = 0; a < ni; a += GEMV_ROWS_PER_WARP) {
                rd.push_back(i);
                rl.push_back(a);
            }
            for (int k = 0; k < h->p[i]; ++k) {
                rdc.push_back(i);
                rlc.push_back(k);
            }
        }
        if constexpr (f64) {
            h->d_gv_l1 = C.up(l1, true);
            h->d_gv_l2 = C.up(l2, true);
        } else {
            h->d_gv_l1_32 = C.up(l1, true);
            h->d_gv_l2_32 = C.up(l2, true);
        }
        h->d_gv_c = C.up(cr, true);
        h->d_g4_desc = C.up(rd, true);
        h->d_g4_row = C.up(rl, true);
        h->n_g4 = (int64_t)rd.size();
        h->d_rd_c = C.up(rdc, true);
        h->d_rl_c = C.up(rlc, true);
        // coarse solve L_E L_E^T e = c: blocked forward / backward substitution
        // with the stored inverses of the diagonal blocks, one cooperative
        // launch (profile figures: the envelope of L_E and L_E^T, the diagonal
        // inverses, once each)
        if (nC > 0) {
            h->d_ctmp = dnew<double>(h, nC);
            h->d_env_row = C.up(h->env_row, true);
            h->d_env_colend = C.up(h->env_colend, true);
            h->coop_blocks = coarse_solve_blocks();
            if (h->coop_blocks <= 0) throw Fail{AMDD_ERR_CUDA};
            const int SB = h->cSB, K = h->cK;
            double el = 0.0, dl = 0.0;
            if (h->cFW == 0)
                for (int64_t r = 0; r < nC; ++r) el += (double)(r - h->env_row[r]) + (double)(h->env_colend[r] - 1 - r);
            for (int k = 0; k < K; ++k) {
                const int r0 = k * SB, r1 = (int)std::min<int64_t>(nC, (int64_t)r0 + SB);
                const double sb = (double)(r1 - r0);
                dl += sb * (sb + 1);
                if (h->cFW > 0) {  // folded: the dense sb x W and sb x V window blocks F_k, G_k
                    int w0 = r0, w1 = r1;
                    for (int r = r0; r < r1; ++r) {
                        w0 = std::min(w0, h->env_row[r]);
                        w1 = std::max(w1, h->env_colend[r]);
                    }
                    el += sb * (double)((r0 - w0) + (w1 - r1));
                }
            }
            h->csolve_flops = 2.0 * el + 2.0 * dl;
            h->csolve_bytes = 8.0 * el + 8.0 * dl + 8.0 * 6.0 * nC;
        }
        // prolongation: copies of each unknown in subdomain order, owners
        std::vector<int64_t> scp(n + 1, 0);
        for (int64_t t = 0; t < h->sum_ni; ++t) scp[omega[t] + 1]++;
        for (int64_t g = 0; g < n; ++g) scp[g + 1] += scp[g];
        std::vector<int32_t> sci(h->sum_ni);
        std::vector<int64_t> fill(scp.begin(), scp.end() - 1);
        for (int64_t t = 0; t < h->sum_ni; ++t) sci[fill[omega[t]]++] = (int32_t)t;
        std::vector<int32_t> og, osub, oa;
        og.reserve(n);
        osub.reserve(n);
        oa.reserve(n);
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < h->nI[i]; ++a) {
                og.push_back(Il[i][a]);
                osub.push_back(i);
                oa.push_back(a);
            }
        h->d_sc_ptr = C.up(scp, true);
        h->d_sc_idx = C.up(sci, true);
        h->d_order_g = C.up(og, true);
        h->d_own_sub = C.up(osub, true);
        h->d_own_a = C.up(oa, true);
        // PCG vectors
        h->d_r = dnew<double>(h, n);
        h->d_z = dnew<double>(h, n);
        h->d_pv = dnew<double>(h, n);
        h->d_q = dnew<double>(h, n);
        h->d_part = dnew<double>(h, DOT_BLOCKS);
        h->d_sc = dnew<PcgScal>(h, 1);
    }
    ck(cudaGetLastError());
    const int e = read_err(h);
    if (e) throw Fail{err_status(e)};
}

// Local solves of the Schwarz methods: rloc = R_i r for every subdomain,
// then y_i = L_i^{-T} L_i^{-1} rloc_i (into d_yloc, or d_yloc32 in the mixed
// form, whose local solves run in FP32).
// The sparse local solves on nb gathered vectors (ld apart) of precision T.
template <typename T>
void sparse_local_solves(amdd_handle* h, const T* rloc, T* yloc, int nb, int64_t ld) {
    const double nnz = (double)h->sl_nnz;
    PScope ps(h, PK_SPLOCAL, 4.0 * nnz * nb,
              nnz * (sizeof(T) + 2.0) + (4.0 + 2.0 * sizeof(T)) * h->sum_ni * nb);
    const size_t smem = h->sl_smem + (size_t)nb * h->sl_nmax * sizeof(T);
    launch_sparse_local_solve<T>(h->d_sl_desc, h->N, smem, h->d_sl_colptr, h->d_sl_row,
                                 static_cast<const T*>(h->d_sl_val), h->d_sl_perm, rloc, yloc, nb, ld, h->s);
}

void local_solves(amdd_handle* h, const double* r) {
    cudaStream_t s = h->s;
    const double tri = (double)h->apply_tri_elems;  // elements of the lower + upper local factors
    {
        PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->sum_ni);
        launch_gather_vec(h->d_omega, h->sum_ni, r, h->d_rloc, s);
    }
    if (h->sparse_local) {
        if (h->precision == 0) {
            sparse_local_solves<double>(h, h->d_rloc, h->d_yloc, 1, h->sum_ni);
        } else {
            {
                PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * h->sum_ni);
                launch_convert<double, float>(h->d_rloc, h->d_rloc32, h->sum_ni, s);
            }
            sparse_local_solves<float>(h, h->d_rloc32, h->d_yloc32, 1, h->sum_ni);
        }
        return;
    }
    if (h->precision == 0) {
        {
            PScope ps(h, PK_GEMV, tri, 8.0 * tri / 2 + 24.0 * h->sum_ni);
            launch_gemv_rows4<double>(h->d_gv_l1, h->d_g4_desc, h->d_g4_row, h->n_g4, s);
        }
        {
            PScope ps(h, PK_GEMV, tri, 8.0 * tri / 2 + 24.0 * h->sum_ni);
            launch_gemv_rows4<double>(h->d_gv_l2, h->d_g4_desc, h->d_g4_row, h->n_g4, s);
        }
    } else {
        // mixed form: local solves in FP32 (FP32 factors, FP32 accumulation)
        {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * h->sum_ni);
            launch_convert<double, float>(h->d_rloc, h->d_rloc32, h->sum_ni, s);
        }
        {
            PScope ps(h, PK_GEMV_F32, tri, 4.0 * tri / 2 + 12.0 * h->sum_ni);
            launch_gemv_rows4<float>(h->d_gv_l1_32, h->d_g4_desc, h->d_g4_row, h->n_g4, s);
        }
        {
            PScope ps(h, PK_GEMV_F32, tri, 4.0 * tri / 2 + 12.0 * h->sum_ni);
            launch_gemv_rows4<float>(h->d_gv_l2_32, h->d_g4_desc, h->d_g4_row, h->n_g4, s);
        }
    }
}

// Coarse correction R_0^T E^{-1} R_0 r of Eq. (two_level_schwarz) from the
// gathered rloc (its Omega_Ii entries): c = Z^T r, the solve with L_E, and
// zc = Z e in owner order (d_zc).  Needs nC > 0.
void inner_coarse_solve(amdd_handle* h);

// the folded form of the coarse solve when the setup built it
void fold_args(const amdd_handle* h, CoarseSolveArgs& a) {
    a.F = h->d_cF;
    a.G = h->d_cG;
    a.fw0 = h->d_cfw0;
    a.gw1 = h->d_cgw1;
    a.FW = h->cFW;
}

void coarse_correction(amdd_handle* h) {
    cudaStream_t s = h->s;
    const double zt = (double)h->sum_zt;
    {
        PScope ps(h, PK_GEMV, 2.0 * zt, 8.0 * zt + 8.0 * h->sum_ni + 16.0 * h->nC);
        launch_gemv_rows<double>(h->d_gv_c, h->d_rd_c, h->d_rl_c, h->nC, s);
    }
    if (h->next) {
        inner_coarse_solve(h);  // multilevel form: e ~ E^{-1} c by GMRES on the next level
    } else {
        double* cin = h->d_c;
        double* eout = h->d_e;
        if (h->d_cperm) {  // the factorisation order of the coarse unknowns
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->nC);
            launch_perm_gather(h->nC, h->d_cperm, h->d_c, h->d_cp, 1, h->nC, s);
            cin = h->d_cp;
            eout = h->d_ep;
        }
        {
            CoarseSolveArgs a{h->d_YE, h->d_YEt, h->d_Yd, h->d_Ydt, h->d_env_row, h->d_env_colend,
                              cin, h->d_ctmp, eout, (int)h->nC, (int)h->nC, h->cSB, h->cK};
            fold_args(h, a);
            PScope ps(h, PK_CSOLVE, h->csolve_flops, h->csolve_bytes);
            ck(launch_coarse_solve(a, h->coop_blocks, s));
        }
        if (h->d_cperm) {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->nC);
            launch_perm_scatter(h->nC, h->d_cperm, h->d_ep, h->d_e, 1, h->nC, s);
        }
    }
    {
        PScope ps(h, PK_GEMV, 2.0 * zt, 8.0 * zt + 8.0 * h->nC + 8.0 * h->n);
        launch_gemv_rows<double>(h->d_gv_zp, h->d_rd_zp, h->d_rl_zp, h->n_zp, s);
    }
}

// z = M^{-1} r, Eq. (two_level_schwarz): one-level sum plus the coarse term,
// summed per unknown in a fixed order.
void apply_one(amdd_handle* h, const double* r, double* z) {
    cudaStream_t s = h->s;
    local_solves(h, r);
    if (h->nC > 0) coarse_correction(h);
    PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * h->sum_ni + 24.0 * h->n);
    const double* zc = h->nC > 0 ? h->d_zc : nullptr;
    if (h->precision == 0)
        launch_scatter_prolong<double>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_yloc, zc, z, s);
    else
        launch_scatter_prolong<float>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_yloc32, zc, z, s);
}

// Buffers of the deflated and restricted forms, on first use.
void ensure_forms(amdd_handle* h) {
    if (h->d_own_idx) return;
    std::vector<int32_t> own(h->n);
    for (int i = 0; i < h->N; ++i)
        for (int a = 0; a < h->nI[i]; ++a) own[h->off_I[i] + a] = (int32_t)(h->off_om[i] + a);  // [I, G] order
    h->d_own_idx = dnew<int32_t>(h, h->n);
    ck(cudaMemcpyAsync(h->d_own_idx, own.data(), h->n * sizeof(int32_t), cudaMemcpyHostToDevice, h->s));
    h->d_zg = dnew<double>(h, h->n);
    h->d_t = dnew<double>(h, h->n);
    ck(cudaStreamSynchronize(h->s));
}

// z = M^{-1} r for the forms of amdd_form:
//   AMDD_FORM_ADDITIVE  Eq. (two_level_schwarz);
//   AMDD_FORM_DEFLATED  Sec. 4.1: zc + M_RAS (r - A zc), zc = R_0^T E^{-1} R_0 r;
//   AMDD_FORM_RAS       Sec. 4.1: sum_i R_i^T D_i A_ii^{-1} R_i r;
//   AMDD_FORM_ASM       sum_i R_i^T A_ii^{-1} R_i r (one-level additive).
void apply_form(amdd_handle* h, int form, const double* r, double* z) {
    if (form == AMDD_FORM_ADDITIVE) {
        apply_one(h, r, z);
        return;
    }
    cudaStream_t s = h->s;
    const bool coarse = form == AMDD_FORM_DEFLATED && h->nC > 0;
    const double* x = r;
    if (form != AMDD_FORM_ASM) ensure_forms(h);
    if (coarse) {
        {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->sum_ni);
            launch_gather_vec(h->d_omega, h->sum_ni, r, h->d_rloc, s);
        }
        coarse_correction(h);
        {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 24.0 * h->n);
            launch_owner_to_global(h->n, h->d_order_g, h->d_zc, h->d_zg, s);
        }
        {
            PScope ps(h, PK_SPMV, 2.0 * h->nnz, 12.0 * h->nnz + 8.0 * (h->n + 1) + 24.0 * h->n);
            launch_spmv_resid(h->n, h->rowptr, h->col, h->val, h->d_zg, r, h->d_t, h->spmv_group, s);
        }
        x = h->d_t;
    }
    local_solves(h, x);
    const double* zc = coarse ? h->d_zc : nullptr;
    if (form == AMDD_FORM_ASM) {
        PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * h->sum_ni + 16.0 * h->n);
        if (h->precision == 0)
            launch_scatter_prolong<double>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_yloc, nullptr, z, s);
        else
            launch_scatter_prolong<float>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_yloc32, nullptr, z, s);
        return;
    }
    PScope ps(h, PK_GATHER_SCATTER, 0.0, (h->precision == 0 ? 8.0 : 4.0) * h->n + (coarse ? 24.0 : 16.0) * h->n);
    if (h->precision == 0)
        launch_ras_prolong<double>(h->n, h->d_order_g, h->d_own_idx, h->d_yloc, zc, z, s);
    else
        launch_ras_prolong<float>(h->n, h->d_order_g, h->d_own_idx, h->d_yloc32, zc, z, s);
}

// Launch wrappers of the PCG loop with their profile accounting.
void spmv_h(amdd_handle* h, const double* x, double* y) {
    PScope ps(h, PK_SPMV, 2.0 * h->nnz, 12.0 * h->nnz + 8.0 * (h->n + 1) + 16.0 * h->n);
    launch_spmv(h->n, h->rowptr, h->col, h->val, x, y, h->spmv_group, h->s);
}
void dot_h(amdd_handle* h, const double* x, const double* y, int which, double tol2) {
    {
        PScope ps(h, PK_PCG_VEC, 2.0 * h->n, 16.0 * h->n);
        launch_dot_partials(h->n, x, y, h->d_part, h->s);
    }
    PScope ps(h, PK_PCG_VEC);
    launch_dot_finalize(h->d_part, h->d_sc, which, tol2, h->s);
}

// Buffers and descriptors of the batched path (MAXB right-hand sides), on first use.
template <typename T>
void* make_local_descs(amdd_handle* h, T* rloc, T* tloc, T* yloc, int which) {
    const int N = h->N;
    std::vector<GemvDescT<T>> g(N);
    for (int i = 0; i < N; ++i) {
        const int ni = h->ni[i];
        if (which == 1)
            g[i] = {static_cast<const T*>(h->lm1[i]), ni, ni, ni, 1, rloc + h->off_om[i], tloc + h->off_om[i]};
        else
            g[i] = {static_cast<const T*>(h->lm2[i]), ni, ni, ni, 2, tloc + h->off_om[i], yloc + h->off_om[i]};
    }
    GemvDescT<T>* d = dnew<GemvDescT<T>>(h, N);
    ck(cudaMemcpyAsync(d, g.data(), N * sizeof(GemvDescT<T>), cudaMemcpyHostToDevice, h->s));
    ck(cudaStreamSynchronize(h->s));
    return d;
}

void ensure_multi(amdd_handle* h) {
    if (h->mb_cap >= MAXB) return;
    const int64_t L = (int64_t)MAXB * h->sum_ni, V = (int64_t)MAXB * h->n, CC = (int64_t)MAXB * std::max<int64_t>(h->nC, 1);
    h->d_m_rloc = dnew<double>(h, L);
    if (h->precision == 0) {
        h->d_m_tloc = dnew<double>(h, L);
        h->d_m_yloc = dnew<double>(h, L);
        h->d_m_gv_l1 = make_local_descs<double>(h, h->d_m_rloc, h->d_m_tloc, h->d_m_yloc, 1);
        h->d_m_gv_l2 = make_local_descs<double>(h, h->d_m_rloc, h->d_m_tloc, h->d_m_yloc, 2);
    } else {
        h->d_m_rloc32 = dnew<float>(h, L);
        h->d_m_tloc32 = dnew<float>(h, L);
        h->d_m_yloc32 = dnew<float>(h, L);
        h->d_m_gv_l1 = make_local_descs<float>(h, h->d_m_rloc32, h->d_m_tloc32, h->d_m_yloc32, 1);
        h->d_m_gv_l2 = make_local_descs<float>(h, h->d_m_rloc32, h->d_m_tloc32, h->d_m_yloc32, 2);
    }
    h->d_m_c = dnew<double>(h, CC);
    h->d_m_ctmp = dnew<double>(h, CC);
    h->d_m_e = dnew<double>(h, CC);
    if (h->nC > 0) {
        std::vector<GemvDesc> cr(h->N);
        for (int i = 0; i < h->N; ++i)
            cr[i] = {h->d_Zt + h->off_zt[i], h->p[i], h->nI[i], h->nI[i], 0, h->d_m_rloc + h->off_om[i],
                     h->d_m_c + h->coff[i]};
        h->d_m_gv_c = dnew<GemvDesc>(h, h->N);
        ck(cudaMemcpyAsync(h->d_m_gv_c, cr.data(), h->N * sizeof(GemvDesc), cudaMemcpyHostToDevice, h->s));
        h->d_m_zc = dnew<double>(h, (int64_t)MAXB * h->n);
        ck(cudaMemsetAsync(h->d_m_zc, 0, (size_t)MAXB * h->n * sizeof(double), h->s));
        std::vector<GemvDesc> zp = h->gv_zp_h;
        int q = 0;
        for (int i = 0; i < h->N; ++i) {
            if (h->p[i] == 0) continue;
            zp[q].x = h->d_m_e + h->coff[i];
            zp[q].y = h->d_m_zc + h->off_I[i];
            ++q;
        }
        h->d_m_gv_zp = dnew<GemvDesc>(h, std::max<int64_t>(q, 1));
        ck(cudaMemcpyAsync(h->d_m_gv_zp, zp.data(), q * sizeof(GemvDesc), cudaMemcpyHostToDevice, h->s));
    }
    h->d_m_q = dnew<double>(h, V);
    h->d_m_r = dnew<double>(h, V);
    h->d_m_z = dnew<double>(h, V);
    h->d_m_p = dnew<double>(h, V);
    h->d_m_part = dnew<double>(h, (int64_t)MAXB * DOT_BLOCKS);
    h->d_m_sc = dnew<PcgScal>(h, MAXB);
    ck(cudaStreamSynchronize(h->s));
    h->mb_cap = MAXB;
}

// z_k = M^{-1} r_k for nb <= MAXB right-hand sides (vectors n apart): every
// factor, Z_i and L_E entry is read once per pass for all of them.
void apply_multi(amdd_handle* h, const double* r, double* z, int nb) {
    if (h->next) {  // inexact coarse solves run one right-hand side at a time
        for (int k = 0; k < nb; ++k) apply_one(h, r + (size_t)k * h->n, z + (size_t)k * h->n);
        return;
    }
    ensure_multi(h);
    cudaStream_t s = h->s;
    const int64_t L = h->sum_ni;
    const double tri = (double)h->apply_tri_elems;
    {
        PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * L * nb);
        launch_gather_vec_multi(h->d_omega, L, r, h->n, h->d_m_rloc, nb, s);
    }
    if (h->sparse_local) {
        if (h->precision == 0) {
            sparse_local_solves<double>(h, h->d_m_rloc, h->d_m_yloc, nb, L);
        } else {
            {
                PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * L * nb);
                launch_convert<double, float>(h->d_m_rloc, h->d_m_rloc32, L * nb, s);
            }
            sparse_local_solves<float>(h, h->d_m_rloc32, h->d_m_yloc32, nb, L);
        }
    } else if (h->precision == 0) {
        auto g1 = static_cast<const GemvDesc*>(h->d_m_gv_l1);
        auto g2 = static_cast<const GemvDesc*>(h->d_m_gv_l2);
        {
            PScope ps(h, PK_GEMV, tri * nb, 8.0 * tri / 2 + 24.0 * L * nb);
            launch_gemv_rows4_multi<double>(g1, h->d_g4_desc, h->d_g4_row, h->n_g4, nb, L, L, s);
        }
        {
            PScope ps(h, PK_GEMV, tri * nb, 8.0 * tri / 2 + 24.0 * L * nb);
            launch_gemv_rows4_multi<double>(g2, h->d_g4_desc, h->d_g4_row, h->n_g4, nb, L, L, s);
        }
    } else {
        auto g1 = static_cast<const GemvDescT<float>*>(h->d_m_gv_l1);
        auto g2 = static_cast<const GemvDescT<float>*>(h->d_m_gv_l2);
        {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 12.0 * L * nb);
            launch_convert<double, float>(h->d_m_rloc, h->d_m_rloc32, L * nb, s);
        }
        {
            PScope ps(h, PK_GEMV_F32, tri * nb, 4.0 * tri / 2 + 12.0 * L * nb);
            launch_gemv_rows4_multi<float>(g1, h->d_g4_desc, h->d_g4_row, h->n_g4, nb, L, L, s);
        }
        {
            PScope ps(h, PK_GEMV_F32, tri * nb, 4.0 * tri / 2 + 12.0 * L * nb);
            launch_gemv_rows4_multi<float>(g2, h->d_g4_desc, h->d_g4_row, h->n_g4, nb, L, L, s);
        }
    }
    if (h->nC > 0) {
        const double zt = (double)h->sum_zt;
        {
            PScope ps(h, PK_GEMV, 2.0 * zt * nb, 8.0 * zt + (8.0 * L + 16.0 * h->nC) * nb);
            launch_gemv_rows_multi<double>(h->d_m_gv_c, h->d_rd_c, h->d_rl_c, h->nC, nb, L, h->nC, s);
        }
        double* cin = h->d_m_c;
        double* eout = h->d_m_e;
        if (h->d_cperm) {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->nC * nb);
            launch_perm_gather(h->nC, h->d_cperm, h->d_m_c, h->d_cp, nb, h->nC, s);
            cin = h->d_cp;
            eout = h->d_ep;
        }
        CoarseSolveArgs a{h->d_YE, h->d_YEt, h->d_Yd, h->d_Ydt, h->d_env_row, h->d_env_colend,
                          cin, h->d_m_ctmp, eout, (int)h->nC, (int)h->nC, h->cSB, h->cK};
        fold_args(h, a);
        a.nb = nb;
        a.ldv = h->nC;
        {
            PScope ps(h, PK_CSOLVE, h->csolve_flops * nb, h->csolve_bytes);
            ck(launch_coarse_solve(a, h->coop_blocks, s));
        }
        if (h->d_cperm) {
            PScope ps(h, PK_GATHER_SCATTER, 0.0, 20.0 * h->nC * nb);
            launch_perm_scatter(h->nC, h->d_cperm, h->d_ep, h->d_m_e, nb, h->nC, s);
        }
        PScope ps(h, PK_GEMV, 2.0 * zt * nb, 8.0 * zt + (8.0 * h->nC + 8.0 * h->n) * nb);
        launch_gemv_rows_multi<double>(h->d_m_gv_zp, h->d_rd_zp, h->d_rl_zp, h->n_zp, nb, h->nC, h->n, s);
    }
    PScope ps(h, PK_GATHER_SCATTER, 0.0, (12.0 * L + 24.0 * h->n) * nb);
    const double* zc = h->nC > 0 ? h->d_m_zc : nullptr;
    if (h->precision == 0)
        launch_scatter_prolong<double>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_m_yloc, zc, z, s, nb, L,
                                       h->n, h->n);
    else
        launch_scatter_prolong<float>(h->n, h->d_order_g, h->d_sc_ptr, h->d_sc_idx, h->d_m_yloc32, zc, z, s, nb, L,
                                      h->n, h->n);
}

void spmv_multi_h(amdd_handle* h, const double* x, double* y, int nb) {
    PScope ps(h, PK_SPMV, 2.0 * h->nnz * nb, 12.0 * h->nnz + 8.0 * (h->n + 1) + 16.0 * h->n * nb);
    launch_spmv_multi(h->n, h->rowptr, h->col, h->val, x, y, nb, h->n, h->s);
}

void dot_multi_h(amdd_handle* h, const double* x, const double* y, int which, double tol2, int nb, int skip) {
    {
        PScope ps(h, PK_PCG_VEC, 2.0 * h->n * nb, 16.0 * h->n * nb);
        launch_dot_partials(h->n, x, y, h->d_m_part, h->s, nb, h->n);
    }
    PScope ps(h, PK_PCG_VEC);
    launch_dot_finalize(h->d_m_part, h->d_m_sc, which, tol2, h->s, nb, skip);
}

// nb <= MAXB independent PCG solves advanced together (one SpMV and one
// batched apply per iteration for all); a converged right-hand side keeps
// its x, r, p.  Returns whether all converged; fills the iteration count and
// the step lengths / ratios of the first right-hand side.
bool pcg_multi(amdd_handle* h, const double* b, double* x, int nb, double rtol, int maxit, int* its0,
               std::vector<double>& al, std::vector<double>& be, PcgScal* sc0) {
    ensure_multi(h);
    cudaStream_t s = h->s;
    const int64_t n = h->n, V = n * nb;
    const double tol2 = rtol * rtol;
    ck(cudaMemsetAsync(h->d_m_sc, 0, nb * sizeof(PcgScal), s));
    spmv_multi_h(h, x, h->d_m_q, nb);
    {
        PScope ps(h, PK_PCG_VEC, 2.0 * V, 24.0 * V);
        launch_axpby(V, 1.0, b, -1.0, h->d_m_q, h->d_m_r, s);
    }
    dot_multi_h(h, b, b, 3, tol2, nb, 0);
    dot_multi_h(h, h->d_m_r, h->d_m_r, 5, tol2, nb, 0);
    std::vector<PcgScal> sc(nb);
    ck(cudaMemcpyAsync(sc.data(), h->d_m_sc, nb * sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    bool all = true, zero = false;
    for (int k = 0; k < nb; ++k) {
        if (sc[k].bb == 0.0) {  // b_k = 0: x_k = 0, done
            ck(cudaMemsetAsync(x + k * n, 0, n * sizeof(double), s));
            sc[k].conv = 1;
            sc[k].rr = 0.0;
            zero = true;
        }
        if (!(sc[k].bb == 0.0 || sc[k].conv)) all = false;
    }
    if (zero) {
        ck(cudaMemcpyAsync(h->d_m_sc, sc.data(), nb * sizeof(PcgScal), cudaMemcpyHostToDevice, s));
        ck(cudaStreamSynchronize(s));
    }
    int its = 0;
    if (!all) {
        apply_multi(h, h->d_m_r, h->d_m_z, nb);
        dot_multi_h(h, h->d_m_r, h->d_m_z, 4, tol2, nb, 0);
        ck(cudaMemcpyAsync(h->d_m_p, h->d_m_z, V * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (its = 1; its <= maxit; ++its) {
            spmv_multi_h(h, h->d_m_p, h->d_m_q, nb);
            dot_multi_h(h, h->d_m_p, h->d_m_q, 0, tol2, nb, 1);
            {
                PScope ps(h, PK_PCG_VEC, 6.0 * V, 48.0 * V);
                launch_pcg_update_xr(n, x, h->d_m_r, h->d_m_p, h->d_m_q, h->d_m_sc, h->d_m_part, s, nb, n, 1);
            }
            {
                PScope ps(h, PK_PCG_VEC);
                launch_dot_finalize(h->d_m_part, h->d_m_sc, 2, tol2, s, nb, 1);
            }
            ck(cudaMemcpyAsync(sc.data(), h->d_m_sc, nb * sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            if ((int)al.size() < sc[0].iters) {  // a new step of the first right-hand side
                if (sc[0].iters > 1) be.push_back(sc[0].beta);
                al.push_back(sc[0].alpha);
            }
            all = true;
            for (int k = 0; k < nb; ++k)
                if (!(sc[k].bb == 0.0 || sc[k].conv)) all = false;
            if (all || its == maxit) break;
            apply_multi(h, h->d_m_r, h->d_m_z, nb);
            dot_multi_h(h, h->d_m_r, h->d_m_z, 1, tol2, nb, 1);
            PScope ps(h, PK_PCG_VEC, 2.0 * V, 24.0 * V);
            launch_pcg_update_p(n, h->d_m_p, h->d_m_z, h->d_m_sc, s, nb, n, 1);
        }
        if (its > maxit) its = maxit;
    }
    *its0 = sc[0].bb == 0.0 ? 0 : sc[0].iters;
    *sc0 = sc[0];
    return all;
}

// GMRES(m) work buffers for restart length m, on first use (grown when a
// later call asks for a longer restart).
void ensure_gmres(amdd_handle* h, int m) {
    if (h->gm_cap >= m) return;
    auto drop = [h](void* p) {
        if (!p) return;
        ck(cudaFreeAsync(p, h->s));
        h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
    };
    drop(h->d_gm_V);
    drop(h->d_gm_Zp);
    const int64_t n = h->n;
    h->gm_ldv = n + (n & 1);  // even: 16-byte aligned vectors for the paired loads
    h->d_gm_V = dnew<double>(h, (int64_t)(m + 1) * h->gm_ldv);
    h->d_gm_Zp = dnew<double>(h, (int64_t)m * h->gm_ldv);
    if (!h->d_gm_st) {
        h->d_gm_wA = dnew<double>(h, n);
        h->d_gm_wB = dnew<double>(h, n);
        h->d_gm_part = dnew<double>(h, (int64_t)(GM_MAXR + 1) * DOT_BLOCKS);
        h->d_gm_st = dnew<GmState>(h, 1);
    }
    h->gm_cap = m;
}

struct GmTail {  // the trailing scalars of GmState, read back after each Arnoldi step
    double bnorm2, beta, hnext, res;
    int conv;
};

struct GmResult {
    int its = 0;
    bool conv = false;
    double res = 0.0;  // |g_{j+1}| / ||b|| at exit
    double bnorm2 = 0.0;
};

// Right-preconditioned GMRES(m) (Saad and Schultz) on A x = b with the
// preconditioner of `form`: Arnoldi on A M with classical Gram-Schmidt
// applied twice, Givens rotations on the Hessenberg matrix,
// x += M V_k y_k at the end of each cycle (the preconditioned vectors
// M v_j are kept), restart from r = b - A x.  Stops when the least-squares
// residual |g_{j+1}| <= rtol ||b||_2 or after maxit Arnoldi steps.
GmResult gmres_run(amdd_handle* h, int form, const double* b, double* x, int m, double rtol, int maxit) {
    ensure_gmres(h, m);
    cudaStream_t s = h->s;
    const int64_t n = h->n;
    double* V = h->d_gm_V;
    const int64_t ldv = h->gm_ldv;
    double* Zp = h->d_gm_Zp;
    double* part = h->d_gm_part;
    GmState* st = h->d_gm_st;
    double* hcol = reinterpret_cast<double*>(reinterpret_cast<char*>(st) + offsetof(GmState, hcol));
    double* H = reinterpret_cast<double*>(reinterpret_cast<char*>(st) + offsetof(GmState, H));
    const char* tail_src = reinterpret_cast<const char*>(st) + offsetof(GmState, bnorm2);
    GmTail tail{};
    GmResult out;
    {
        PScope ps(h, PK_GMRES, 2.0 * n, 8.0 * n);
        launch_dot_partials(n, b, b, part, s);
    }
    {
        PScope ps(h, PK_GMRES);
        launch_gm_norm(part, st, 0, s);
    }
    ck(cudaMemcpyAsync(&tail, tail_src, sizeof(GmTail), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    out.bnorm2 = tail.bnorm2;
    if (tail.bnorm2 == 0.0) {  // b = 0: x = 0
        ck(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        out.conv = true;
        return out;
    }
    out.res = 1.0;
    while (out.its < maxit) {
        // r = b - A x, beta = ||r||, v_0 = r / beta, g = beta e_1
        {
            PScope ps(h, PK_SPMV, 2.0 * h->nnz, 12.0 * h->nnz + 8.0 * (n + 1) + 24.0 * n);
            launch_spmv_resid(n, h->rowptr, h->col, h->val, x, b, V, h->spmv_group, s);
        }
        {
            PScope ps(h, PK_GMRES, 2.0 * n, 8.0 * n);
            launch_dot_partials(n, V, V, part, s);
        }
        {
            PScope ps(h, PK_GMRES);
            launch_gm_norm(part, st, 1, s);
        }
        {
            PScope ps(h, PK_GMRES, (double)n, 16.0 * n);
            launch_gm_scale(n, V, V, st, 0, s);
        }
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = V + (int64_t)j * ldv;
            double* zj = Zp + (int64_t)j * ldv;
            double* vn = V + (int64_t)(j + 1) * ldv;
            double* Hc = H + (int64_t)j * (GM_MAXR + 1);
            const int kk = j + 1;
            apply_form(h, form, vj, zj);
            {
                PScope ps(h, PK_SPMV, 2.0 * h->nnz, 12.0 * h->nnz + 8.0 * (n + 1) + 16.0 * n);
                launch_spmv(n, h->rowptr, h->col, h->val, zj, h->d_gm_wA, h->spmv_group, s);
            }
            // CGS2: h1 = V^T w; w1 = w - V h1, h2 = V^T w1; w2 = w1 - V h2, ||w2||
            {
                PScope ps(h, PK_GMRES, 2.0 * kk * n, 8.0 * (kk + 1) * n);
                launch_gm_ortho(n, V, ldv, kk, nullptr, h->d_gm_wA, nullptr, part, 0, s);
            }
            {
                PScope ps(h, PK_GMRES);
                launch_gm_finalize(part, kk, hcol, Hc, 0, s);
            }
            {
                PScope ps(h, PK_GMRES, 4.0 * kk * n, 8.0 * (kk + 2) * n);
                launch_gm_ortho(n, V, ldv, kk, hcol, h->d_gm_wA, h->d_gm_wB, part, 1, s);
            }
            {
                PScope ps(h, PK_GMRES);
                launch_gm_finalize(part, kk, hcol, Hc, 1, s);
            }
            {
                PScope ps(h, PK_GMRES, (2.0 * kk + 2.0) * n, 8.0 * (kk + 2) * n);
                launch_gm_ortho(n, V, ldv, kk, hcol, h->d_gm_wB, vn, part, 2, s);
            }
            {
                PScope ps(h, PK_GMRES);
                launch_gm_givens(part, st, j, rtol, s);
            }
            {
                PScope ps(h, PK_GMRES, (double)n, 16.0 * n);
                launch_gm_scale(n, vn, vn, st, 1, s);
            }
            ++out.its;
            k = kk;
            ck(cudaMemcpyAsync(&tail, tail_src, sizeof(GmTail), cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            out.res = tail.res;
            if (tail.conv) out.conv = true;
            if (out.conv || out.its >= maxit) break;
        }
        {
            PScope ps(h, PK_GMRES);
            launch_gm_trisolve(st, k, s);
        }
        {
            PScope ps(h, PK_GMRES, 2.0 * k * n, 8.0 * (k + 2) * n);
            launch_gm_combine(n, Zp, ldv, k, st, x, s);
        }
        if (out.conv) break;
    }
    return out;
}

// Inexact coarse solve of the multilevel form: GMRES on E e = c (the next
// level's operator) from e = 0, preconditioned by the next level's deflated
// form.
void inner_coarse_solve(amdd_handle* h) {
    ck(cudaMemsetAsync(h->d_e, 0, h->nC * sizeof(double), h->s));
    const GmResult g = gmres_run(h->next, AMDD_FORM_DEFLATED, h->d_c, h->d_e, h->in_restart, h->in_rtol, h->in_maxit);
    h->in_calls += 1;
    h->in_its += g.its;
    h->in_max = std::max(h->in_max, g.its);
}

// Whether single right-hand-side PCG iterations may run as a graph: asked
// for, no inexact coarse solve on a next level (it synchronises with the
// host), and no profiling events around the loop's kernel classes.
bool graph_ok(const amdd_handle* h) {
    if (!h->use_graphs || h->pg_failed || h->next) return false;
    if (h->prof.on) {
        const uint32_t loop = (1u << PK_SPMV) | (1u << PK_GEMV) | (1u << PK_GEMV_F32) | (1u << PK_GATHER_SCATTER) |
                              (1u << PK_PCG_VEC) | (1u << PK_CSOLVE);
        if (h->prof.mask & loop) return false;
    }
    return true;
}

// The PCG loop as one graph, built once per handle and tolerance:
//   while (not converged and iterations < maxit) {
//       z = M^{-1} r;  rz' = r.z, beta = rz' / rz, rz = rz';  p = z + beta p;
//       q = A p;  alpha = rz / p.q;  x += alpha p, r -= alpha q;  rr = r.r
//   }
// on the handle's vectors (x accumulates in d_px), the condition set on the
// device after each pass (pcg_loop_cond_kernel), so a whole solve is one
// graph launch and one synchronisation.  The same kernels in the same order
// as the per-iteration loop, so the results are the same bits.  Returns false
// when the runtime cannot capture or instantiate it (the solve then launches
// iteration by iteration).
bool pcg_graph(amdd_handle* h, double tol2, int maxit) {
    if (h->pg_exec && h->pg_tol2 == tol2 && maxit <= h->pg_cap) return true;
    if (h->pg_exec) cudaGraphExecDestroy(h->pg_exec);
    if (h->pg_graph) cudaGraphDestroy(h->pg_graph);
    h->pg_exec = nullptr;
    h->pg_graph = nullptr;
    const int64_t n = h->n;
    cudaStream_t s = h->s;
    cudaStream_t s_main = h->s;
    if (maxit > h->pg_cap) {
        h->pg_cap = std::max(maxit, 1024);
        h->d_alog = dnew<double>(h, h->pg_cap);
        h->d_blog = dnew<double>(h, h->pg_cap);
    }
    if (!h->d_px) h->d_px = dnew<double>(h, n);
    if (!h->d_maxit) h->d_maxit = dnew<int>(h, 1);
    ck(cudaStreamSynchronize(s));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaGraphConditionalHandle loop{};
    cudaGraphNodeParams cp{};
    cudaGraphNode_t node = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    // capture on a private non-blocking stream: the handle's stream may be the
    // legacy default stream, which cannot be captured; every launch of the
    // loop goes to h->s, so h->s names the capture stream meanwhile
    if (ok && !h->s_cap) ok = cudaStreamCreateWithFlags(&h->s_cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok)
        ok = cudaStreamBeginCaptureToGraph(h->s_cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        bool launched = true;
        h->s = h->s_cap;
        s = h->s_cap;
        try {
            apply_one(h, h->d_r, h->d_z);
            dot_h(h, h->d_r, h->d_z, 1, tol2);
            launch_pcg_update_p(n, h->d_pv, h->d_z, h->d_sc, s);
            spmv_h(h, h->d_pv, h->d_q);
            dot_h(h, h->d_pv, h->d_q, 0, tol2);
            launch_pcg_update_xr(n, h->d_px, h->d_r, h->d_pv, h->d_q, h->d_sc, h->d_part, s);
            launch_dot_finalize(h->d_part, h->d_sc, 2, tol2, s);
            launch_pcg_loop_cond(h->d_sc, h->d_maxit, h->d_alog, h->d_blog, loop, s);
        } catch (...) {
            launched = false;
        }
        cudaGraph_t body = nullptr;
        const cudaError_t e = cudaStreamEndCapture(h->s_cap, &body);
        h->s = s_main;
        s = s_main;
        ok = launched && e == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        h->pg_failed = true;
        return false;
    }
    h->pg_graph = g;
    h->pg_exec = ex;
    h->pg_tol2 = tol2;
    return true;
}

amdd_status guard_exc() {
    try {
        throw;
    } catch (const Fail& f) {
        return f.st;
    } catch (const std::bad_alloc&) {
        return AMDD_ERR_OOM;
    } catch (...) {
        return AMDD_ERR_CUDA;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

amdd_status amdd_opts_default(amdd_opts* o) {
    if (!o) return AMDD_ERR_INVALID;
    std::memset(o, 0, sizeof(*o));
    o->eps = std::ldexp(1.0, -52);
    o->max_sweeps = 60;
    o->tie_band = 1e-10;
    o->use_graphs = 1;
    o->autotune = 1;
    o->tensor_cores = 1;
    return AMDD_OK;
}

amdd_status amdd_gemm_f32(int32_t m, int32_t n, int32_t k, float alpha, const float* A, int32_t lda, int32_t ta,
                          const float* B, int32_t ldb, int32_t tb, float beta, float* C, int32_t ldc,
                          int32_t tensor_cores, void* stream) {
    if (m < 0 || n < 0 || k < 0 || (ta != 0 && ta != 1) || (tb != 0 && tb != 1) ||
        (tensor_cores != 0 && tensor_cores != 1))
        return AMDD_ERR_INVALID;
    if (m == 0 || n == 0) return AMDD_OK;
    if (!C || (k > 0 && (!A || !B)) || ldc < n || (k > 0 && lda < (ta ? m : k)) || (k > 0 && ldb < (tb ? k : n)))
        return AMDD_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GemmDescT<float> g;
    g.A = A;
    g.B = B;
    g.C = C;
    g.m = m;
    g.n = n;
    g.k = k;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.ta = ta;
    g.tb = tb;
    g.lower = 0;
    g.kfrom_row = 0;
    g.alpha = alpha;
    g.beta = beta;
    const int tile = tensor_cores ? TC_GEMM_TILE : GEMM_T;
    std::vector<TileRef> tiles;
    for (int a = 0; a < cdiv(m, tile); ++a)
        for (int b = 0; b < cdiv(n, tile); ++b) tiles.push_back({0, a, b});
    void* buf = nullptr;
    const size_t bytes = sizeof(g) + tiles.size() * sizeof(TileRef) + sizeof(int);
    if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return AMDD_ERR_OOM;
    }
    std::vector<unsigned char> host(bytes, 0);
    std::memcpy(host.data(), &g, sizeof(g));
    std::memcpy(host.data() + sizeof(g), tiles.data(), tiles.size() * sizeof(TileRef));
    auto* dg = static_cast<GemmDescT<float>*>(buf);
    auto* dt = reinterpret_cast<TileRef*>(static_cast<unsigned char*>(buf) + sizeof(g));
    auto* derr = reinterpret_cast<int*>(static_cast<unsigned char*>(buf) + sizeof(g) + tiles.size() * sizeof(TileRef));
    amdd_status st = AMDD_OK;
    if (cudaMemcpyAsync(buf, host.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) st = AMDD_ERR_CUDA;
    if (st == AMDD_OK) {
        if (tensor_cores)
            launch_gemm_tc(dg, dt, (int)tiles.size(), derr, s);
        else
            launch_gemm<float>(dg, dt, (int)tiles.size(), tile, s);
        int e = 0;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = AMDD_ERR_CUDA;
        else if (e)
            st = err_status(e);
    }
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    return st;
}

amdd_status amdd_wait_selftest(int32_t set_flag, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* buf = nullptr;  // flag, error word
    if (cudaMallocAsync((void**)&buf, 2 * sizeof(int), s) != cudaSuccess) return AMDD_ERR_OOM;
    const int init[2] = {set_flag ? 1 : 0, 0};
    int err = 0;
    cudaMemcpyAsync(buf, init, sizeof(init), cudaMemcpyHostToDevice, s);
    launch_wait_selftest(buf, 4000000ll, buf + 1, s);  // about 2 ms at 2 GHz
    cudaMemcpyAsync(&err, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return AMDD_ERR_CUDA;
    return err & DERR_TIMEOUT ? AMDD_ERR_TIMEOUT : AMDD_OK;
}

amdd_status amdd_spmv(const amdd_csr* A, const double* x, double* y, void* stream) {
    if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->rowptr || !x || !y)) || (A->nnz > 0 && (!A->colind || !A->val)))
        return AMDD_ERR_INVALID;
    if (A->n > INT32_MAX) return AMDD_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_spmv(A->n, A->rowptr, A->colind, A->val, x, y, spmv_group_for(A->n, A->nnz), s);
    if (cudaGetLastError() != cudaSuccess) return AMDD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMDD_ERR_CUDA;
    return AMDD_OK;
}

amdd_status amdd_overlap_sets(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* part,
                              int32_t i, int32_t overlap, int32_t* I, int32_t capI, int32_t* G, int32_t capG,
                              int32_t* D, int32_t capD, int32_t* nI, int32_t* nG, int32_t* nD) {
    if (n < 1 || n > INT32_MAX || !rowptr || !colind || !part || i < 0 || overlap < 0) return AMDD_ERR_INVALID;
    try {
        const int64_t nnz = rowptr[n];
        if (rowptr[0] != 0 || nnz < 0) return AMDD_ERR_INVALID;
        for (int64_t r = 0; r < n; ++r)
            if (rowptr[r] > rowptr[r + 1]) return AMDD_ERR_INVALID;
        for (int64_t k = 0; k < nnz; ++k)
            if (colind[k] < 0 || colind[k] >= n) return AMDD_ERR_INVALID;
        std::vector<int32_t> Iv;
        for (int64_t g = 0; g < n; ++g)
            if (part[g] == i) Iv.push_back((int32_t)g);
        std::vector<int32_t> mark(n, -1), Gv, Dv;
        overlap_layers(rowptr, colind, Iv, overlap, i, mark.data(), Gv, Dv);
        if (nI) *nI = (int32_t)Iv.size();
        if (nG) *nG = (int32_t)Gv.size();
        if (nD) *nD = (int32_t)Dv.size();
        if ((I && capI < (int64_t)Iv.size()) || (G && capG < (int64_t)Gv.size()) || (D && capD < (int64_t)Dv.size()))
            return AMDD_ERR_INVALID;
        if (I) std::copy(Iv.begin(), Iv.end(), I);
        if (G) std::copy(Gv.begin(), Gv.end(), G);
        if (D) std::copy(Dv.begin(), Dv.end(), D);
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

amdd_status amdd_setup(const amdd_csr* A, const int32_t* part, int32_t N, int32_t overlap, double tau,
                       const amdd_opts* opts, void* stream, amdd_handle** out) {
    if (!out) return AMDD_ERR_INVALID;
    *out = nullptr;
    if (!A || !part || N < 1 || overlap < 1 || !(tau > 0.0) || A->n < 1 || A->nnz < A->n || !A->rowptr ||
        !A->colind || !A->val || N > A->n || A->n > INT32_MAX)
        return AMDD_ERR_INVALID;
    amdd_opts o;
    amdd_opts_default(&o);
    if (opts) {
        o = *opts;
        if (!(o.eps > 0.0) || o.max_sweeps < 1 || o.precision < 0 || o.precision > 2) return AMDD_ERR_INVALID;
        if (o.reserved != 0 || o.keep_coarse_matrix < 0 || o.keep_coarse_matrix > 1) return AMDD_ERR_INVALID;
        if (!(o.tie_band >= 0.0) || o.use_graphs < 0 || o.use_graphs > 1 || o.autotune < 0 || o.autotune > 1)
            return AMDD_ERR_INVALID;
        if (o.tensor_cores < 0 || o.tensor_cores > 1) return AMDD_ERR_INVALID;
        if (o.local_solver < 0 || o.local_solver > 2) return AMDD_ERR_INVALID;
        if (o.jacobi_inner_sweeps < 0 || o.jacobi_inner_sweeps > 64) return AMDD_ERR_INVALID;
        if (o.profile_classes >> PK_COUNT) return AMDD_ERR_INVALID;
        if (o.eig_solver < 0 || o.eig_solver > 3) return AMDD_ERR_INVALID;
        // the matrix-free eigensolve: FP64 only, with the shift far enough above
        // the FP64 rounding for eq. (invAii) not to cancel
        if (o.eig_solver == 3 && (o.precision != 0 || o.eps < 0x1p-30 || o.keep_proposal_data))
            return AMDD_ERR_INVALID;
        if (o.eig_solver == 2 &&
            (!o.proposal || !o.proposal->weights || !o.proposal->mean || !o.proposal->sd))
            return AMDD_ERR_INVALID;
    }
    const auto t0 = std::chrono::steady_clock::now();
    amdd_handle* h = nullptr;
    try {
        h = new amdd_handle();
        h->s = static_cast<cudaStream_t>(stream);
        ck(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
        ck(cudaEventCreateWithFlags(&h->ev_panel, cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&h->ev_far, cudaEventDisableTiming));
        ck(cudaStreamCreateWithFlags(&h->s3, cudaStreamNonBlocking));
        ck(cudaStreamCreateWithFlags(&h->s4, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&h->ev_panel3, &h->ev_far3, &h->ev_spec_in, &h->ev_spec_done})
            ck(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        h->n = A->n;
        h->nnz = A->nnz;
        h->N = N;
        h->overlap = overlap;
        h->tau = tau;
        h->eps = o.eps;
        h->max_sweeps = o.max_sweeps;
        h->prof.on = o.profile != 0;
        h->prof.mask = o.profile_classes ? o.profile_classes : ~0u;
        h->precision = o.precision;
        h->eig_solver = o.eig_solver;
        h->keep_prop = o.keep_proposal_data != 0;
        h->keep_E = o.keep_coarse_matrix;
        h->tie_band = o.tie_band;
        h->mem_budget = o.mem_budget;
        h->use_graphs = o.use_graphs;
        h->autotune = o.autotune;
        h->tensor_cores = o.tensor_cores;
        h->local_solver = o.local_solver;
        h->jacobi_inner = o.jacobi_inner_sweeps ? o.jacobi_inner_sweeps : 1;
        if (o.eig_solver == 2) {
            h->prop = *o.proposal;
            h->have_prop = true;
        }
        if (o.precision == 0)
            do_setup<double, double>(h, A, part);
        else if (o.precision == 1)
            do_setup<float, float>(h, A, part);
        else
            do_setup<float, double>(h, A, part);
        ck(cudaStreamSynchronize(h->s));
    } catch (...) {
        const amdd_status st = guard_exc();
        if (h) {
            cudaStreamSynchronize(h->s);
            amdd_destroy(h);
        }
        return st;
    }
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return AMDD_OK;
}

amdd_status amdd_apply(amdd_handle* h, const double* r, double* z, int32_t nrhs) {
    if (!h || !r || !z || nrhs < 0 || r == z) return AMDD_ERR_INVALID;
    try {
        if (nrhs == 1)
            apply_one(h, r, z);
        else
            for (int k = 0; k < nrhs; k += MAXB)
                apply_multi(h, r + (size_t)k * h->n, z + (size_t)k * h->n, std::min(MAXB, nrhs - k));
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(h->s));
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

namespace {

// Number of eigenvalues below x of the symmetric tridiagonal (d, e) by the
// signs of the LDL^T pivots (Sturm sequence), with a tiny pivot replaced by a
// signed floor so the recurrence never divides by zero.
int tri_count_below(const std::vector<double>& d, const std::vector<double>& e, double x, double floor) {
    int c = 0;
    double q = d[0] - x;
    if (std::fabs(q) < floor) q = -floor;
    if (q < 0.0) ++c;
    for (size_t j = 1; j < d.size(); ++j) {
        q = d[j] - x - e[j - 1] * e[j - 1] / q;
        if (std::fabs(q) < floor) q = -floor;
        if (q < 0.0) ++c;
    }
    return c;
}

// Smallest and largest eigenvalue of the Lanczos tridiagonal of PCG (the
// CG-Lanczos relation): T_11 = 1/alpha_1, T_jj = 1/alpha_j +
// beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j; bisection inside
// the Gershgorin interval to a relative width of 1e-15.
void lanczos_extremes(const std::vector<double>& al, const std::vector<double>& be, double* lo, double* hi) {
    const size_t k = al.size();
    if (k == 0) {
        *lo = *hi = std::numeric_limits<double>::quiet_NaN();
        return;
    }
    std::vector<double> d(k), e(k > 1 ? k - 1 : 1, 0.0);
    for (size_t j = 0; j < k; ++j) d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    for (size_t j = 0; j + 1 < k; ++j) e[j] = std::sqrt(std::max(be[j], 0.0)) / al[j];
    double gl = d[0], gu = d[0];
    for (size_t j = 0; j < k; ++j) {
        const double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < k ? std::fabs(e[j]) : 0.0);
        gl = std::min(gl, d[j] - r);
        gu = std::max(gu, d[j] + r);
    }
    const double scale = std::max(std::fabs(gl), std::fabs(gu));
    const double floor = 1e-300 * std::max(1.0, scale);
    auto kth = [&](int target) {  // smallest x with count_below(x) > target
        double a = gl, b = gu;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
            const double m = 0.5 * (a + b);
            if (tri_count_below(d, e, m, floor) > target)
                b = m;
            else
                a = m;
        }
        return 0.5 * (a + b);
    };
    *lo = kth(0);
    *hi = kth((int)k - 1);
}

}  // namespace

amdd_status amdd_get_eig_iterations(const amdd_handle* h, int32_t* iters, int32_t cap) {
    if (!h || !iters || cap < h->N) return AMDD_ERR_INVALID;
    for (int i = 0; i < h->N; ++i) iters[i] = i < (int)h->eig_iters.size() ? h->eig_iters[i] : -2;
    return AMDD_OK;
}

amdd_status amdd_proposal_export(const amdd_handle* hc, float* feat, float* target, int32_t* sub, int32_t cap,
                                 int32_t* count) {
    if (!hc || !count) return AMDD_ERR_INVALID;
    amdd_handle* h = const_cast<amdd_handle*>(hc);
    if (!h->keep_prop) return AMDD_ERR_INVALID;
    const int np = (int)h->prop_sub.size();
    *count = np;
    if (!feat && !target && !sub) return AMDD_OK;
    if (cap < np) return AMDD_ERR_INVALID;
    if (np == 0) return AMDD_OK;
    try {
        cudaStream_t s = h->s;
        if (feat)
            ck(cudaMemcpyAsync(feat, h->prop_feat, (size_t)np * PROP_NF * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (sub)
            for (int q = 0; q < np; ++q) sub[q] = h->prop_sub[q];
        if (target) {
            // B^T Q Q^T B = G M^{-1} G^T with G = Bt Zt^T (16 x p) and M = Zt Zt^T = L_M L_M^T:
            // H = G L_M^{-T}, target = H H^T
            Ctx C(h);
            std::vector<int64_t> om(np + 1, 0), og(np + 1, 0);
            for (int q = 0; q < np; ++q) {
                const int pq = h->p[h->prop_sub[q]];
                om[q + 1] = om[q] + (int64_t)pq * pq;
                og[q + 1] = og[q] + (int64_t)PROP_NB * pq;
            }
            double* M = C.tnew<double>(om[np]);
            double* Mi = C.tnew<double>(om[np]);
            double* G = C.tnew<double>(og[np]);
            double* H = C.tnew<double>(og[np]);
            double* Q = C.tnew<double>((int64_t)np * PROP_NO);
            int64_t lsz = 0;
            for (int q = 0; q < np; ++q) lsz += (int64_t)cdiv(h->p[h->prop_sub[q]], CHOL_NB) * CHOL_NB * CHOL_NB;
            double* linv = C.tnew<double>(lsz);
            std::vector<GemmDesc> g1, g2;
            std::vector<CholDesc> cd;
            std::vector<TrtriDesc> td;
            int64_t lo = 0;
            for (int q = 0; q < np; ++q) {
                const int i = h->prop_sub[q], pq = h->p[i], nIi = h->nI[i];
                const double* Zt = h->d_Zt + h->off_zt[i];
                g1.push_back(gd(Zt, nIi, 0, Zt, nIi, 1, M + om[q], pq, pq, pq, nIi, 1.0, 0.0, 0));
                g2.push_back(gd(h->prop_bt + h->prop_off_b[q], nIi, 0, Zt, nIi, 1, G + og[q], pq, PROP_NB, pq, nIi, 1.0,
                                0.0, 0));
                cd.push_back({M + om[q], pq, pq, pq, nullptr, linv + lo});
                td.push_back({M + om[q], Mi + om[q], linv + lo, pq, pq, pq});
                lo += (int64_t)cdiv(pq, CHOL_NB) * CHOL_NB * CHOL_NB;
            }
            gemm(C, g1);
            gemm(C, g2);
            chol_batched<double>(C, cd);
            trtri_batched<double>(C, td);
            std::vector<GemmDesc> g3, g4;
            for (int q = 0; q < np; ++q) {
                const int pq = h->p[h->prop_sub[q]];
                g3.push_back(gd(G + og[q], pq, 0, Mi + om[q], pq, 1, H + og[q], pq, PROP_NB, pq, pq, 1.0, 0.0, 0));
                g4.push_back(gd(H + og[q], pq, 0, H + og[q], pq, 1, Q + (int64_t)q * PROP_NO, PROP_NB, PROP_NB, PROP_NB,
                                pq, 1.0, 0.0, 0));
            }
            gemm(C, g3);
            gemm(C, g4);
            std::vector<double> hq((size_t)np * PROP_NO);
            ck(cudaMemcpyAsync(hq.data(), Q, hq.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            {
                const int e = read_err(h);
                if (e) throw Fail{err_status(e)};
            }
            for (size_t t = 0; t < hq.size(); ++t) target[t] = (float)hq[t];
        }
        ck(cudaStreamSynchronize(s));
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

// The MLP entry points run on a transient handle that only carries the
// stream (no profiling), so the batched GEMM and its uploads serve them too.
amdd_status amdd_mlp_sizes(int32_t n, int64_t* nparam, int64_t* nwork) {
    if (n < 1 || !nparam || !nwork) return AMDD_ERR_INVALID;
    *nparam = MLP_NPARAM;
    *nwork = (int64_t)9 * n * PROP_NH + n + 16;
    return AMDD_OK;
}

amdd_status amdd_mlp_feature_stats(const float* feat, int32_t n, float* mean, float* sd, void* stream) {
    if (n < 1 || !feat || !mean || !sd) return AMDD_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_feature_stats(feat, n, mean, sd, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return AMDD_ERR_CUDA;
    return AMDD_OK;
}

amdd_status amdd_mlp_normalize(const float* feat, const float* mean, const float* sd, int32_t n, float* x,
                               void* stream) {
    if (n < 1 || !feat || !mean || !sd || !x) return AMDD_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_normalize_features(feat, mean, sd, x, n, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return AMDD_ERR_CUDA;
    return AMDD_OK;
}

amdd_status amdd_mlp_forward(const float* wb, const float* x, int32_t n, float* q, float* work, void* stream) {
    if (n < 1 || !wb || !x || !q || !work) return AMDD_ERR_INVALID;
    try {
        amdd_handle tmp;
        tmp.s = static_cast<cudaStream_t>(stream);
        {
            Ctx C(&tmp);
            mlp_forward(C, wb, x, n, work, q);
            ck(cudaGetLastError());
            ck(cudaStreamSynchronize(tmp.s));
        }
        ck(cudaStreamSynchronize(tmp.s));
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

amdd_status amdd_mlp_train_step(float* w, float* wb, float* m, float* v, int32_t t, float lr, const float* x,
                                const float* qt, int32_t n, float* grad, float* work, float* loss, void* stream) {
    if (n < 1 || !wb || !x || !qt || !grad || !work || !loss || !(lr >= 0.0f)) return AMDD_ERR_INVALID;
    if (lr > 0.0f && (!w || !m || !v || t < 1)) return AMDD_ERR_INVALID;
    try {
        amdd_handle tmp;
        tmp.s = static_cast<cudaStream_t>(stream);
        {
            Ctx C(&tmp);
            mlp_backward(C, wb, x, qt, n, work, grad, loss);
            if (lr > 0.0f) launch_adam(w, wb, m, v, grad, (int)MLP_NPARAM, lr, t, tmp.s);
            ck(cudaGetLastError());
            ck(cudaStreamSynchronize(tmp.s));
        }
        ck(cudaStreamSynchronize(tmp.s));
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

amdd_status amdd_mlp_round_bf16(const float* w, float* wb, int64_t n, void* stream) {
    if (n < 1 || n > INT32_MAX || !w || !wb) return AMDD_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_bf16_round(w, wb, (int)n, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return AMDD_ERR_CUDA;
    return AMDD_OK;
}

amdd_status amdd_lanczos_extremes(const double* alpha, const double* beta, int32_t k, double* lo, double* hi) {
    if (k < 0 || !lo || !hi || (k > 0 && !alpha) || (k > 1 && !beta)) return AMDD_ERR_INVALID;
    try {
        std::vector<double> al(alpha, alpha + k), be;
        if (k > 1) be.assign(beta, beta + (k - 1));
        for (int j = 0; j < k; ++j)
            if (!(al[j] > 0.0)) return AMDD_ERR_INVALID;
        for (int j = 0; j + 1 < k; ++j)
            if (!(be[j] >= 0.0)) return AMDD_ERR_INVALID;
        lanczos_extremes(al, be, lo, hi);
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

amdd_status amdd_pcg_solve(amdd_handle* h, const double* b, double* x, int32_t nrhs, double rtol, int32_t maxit,
                           amdd_stats* stats) {
    if (!h || !b || !x || nrhs < 0 || !(rtol >= 0.0) || maxit < 0) return AMDD_ERR_INVALID;
    const auto t0 = std::chrono::steady_clock::now();
    amdd_status result = AMDD_OK;
    try {
        cudaStream_t s = h->s;
        const int64_t n = h->n;
        const double tol2 = rtol * rtol;
        // a NaN or infinity in b or in the initial guess: AMDD_ERR_INVALID
        require(all_finite(h, b, (int64_t)nrhs * n) && all_finite(h, x, (int64_t)nrhs * n));
        if (nrhs > 1) {
            // batched independent solves, MAXB right-hand sides per pass
            std::vector<double> al, be;
            PcgScal sc0{};
            int its0 = 0;
            bool conv0 = true;
            for (int k = 0; k < nrhs; k += MAXB) {
                const int nb = std::min(MAXB, nrhs - k);
                std::vector<double> a2, b2;
                PcgScal sck{};
                int itk = 0;
                const bool all = pcg_multi(h, b + (size_t)k * n, x + (size_t)k * n, nb, rtol, maxit, &itk,
                                           k == 0 ? al : a2, k == 0 ? be : b2, &sck);
                if (!all) result = AMDD_ERR_NOCONV;
                if (k == 0) {
                    its0 = itk;
                    sc0 = sck;
                    conv0 = sck.bb == 0.0 || sck.conv;
                }
            }
            if (stats) {
                spmv_h(h, x, h->d_q);
                launch_axpby(n, 1.0, b, -1.0, h->d_q, h->d_z, s);
                dot_h(h, h->d_z, h->d_z, 5, tol2);
                PcgScal st{};
                ck(cudaMemcpyAsync(&st, h->d_sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
                ck(cudaStreamSynchronize(s));
                stats->iterations = its0;
                stats->converged = conv0 ? 1 : 0;
                stats->rel_residual = sc0.bb > 0.0 ? std::sqrt(sc0.rr / sc0.bb) : 0.0;
                stats->true_rel_residual = sc0.bb > 0.0 ? std::sqrt(st.rr / sc0.bb) : 0.0;
                lanczos_extremes(al, be, &stats->ritz_min, &stats->ritz_max);
                stats->cond_est = stats->ritz_max / stats->ritz_min;
            }
            nrhs = 0;  // done
        }
        for (int k = 0; k < nrhs; ++k) {
            const double* bk = b + (size_t)k * n;
            double* xk = x + (size_t)k * n;
            PcgScal sc0{};
            ck(cudaMemcpyAsync(h->d_sc, &sc0, sizeof(PcgScal), cudaMemcpyHostToDevice, s));
            // r = b - A x0
            spmv_h(h, xk, h->d_q);
            {
                PScope ps(h, PK_PCG_VEC, 2.0 * n, 24.0 * n);
                launch_axpby(n, 1.0, bk, -1.0, h->d_q, h->d_r, s);
            }
            dot_h(h, bk, bk, 3, tol2);
            dot_h(h, h->d_r, h->d_r, 5, tol2);
            PcgScal sc{};
            ck(cudaMemcpyAsync(&sc, h->d_sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            int its = 0;
            std::vector<double> al, be;  // PCG step lengths and ratios (condition estimate)
            bool conv = sc.bb == 0.0 || sc.conv;
            if (sc.bb == 0.0) {
                ck(cudaMemsetAsync(xk, 0, n * sizeof(double), s));
                sc.rr = 0.0;
            }
            if (!conv && maxit >= 1 && graph_ok(h) && pcg_graph(h, tol2, maxit)) {
                // p = 0 and rz = 1: the first pass of the loop forms p = z + (r.z / 1) 0 = z
                // exactly, the direction of the first iteration
                static const double one = 1.0;
                ck(cudaMemcpyAsync(h->d_px, xk, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                ck(cudaMemsetAsync(h->d_pv, 0, n * sizeof(double), s));
                ck(cudaMemcpyAsync(reinterpret_cast<char*>(h->d_sc) + offsetof(PcgScal, rz), &one, sizeof(double),
                                   cudaMemcpyHostToDevice, s));
                ck(cudaMemcpyAsync(h->d_maxit, &maxit, sizeof(int), cudaMemcpyHostToDevice, s));
                ck(cudaGraphLaunch(h->pg_exec, s));
                ck(cudaMemcpyAsync(xk, h->d_px, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                ck(cudaMemcpyAsync(&sc, h->d_sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
                ck(cudaStreamSynchronize(s));
                its = sc.iters;
                conv = sc.conv != 0;
                h->graph_solves += 1;
                if (k == 0 && its > 0) {
                    al.resize(its);
                    be.resize(its - 1);
                    ck(cudaMemcpyAsync(al.data(), h->d_alog, its * sizeof(double), cudaMemcpyDeviceToHost, s));
                    if (its > 1)
                        ck(cudaMemcpyAsync(be.data(), h->d_blog, (its - 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                           s));
                    ck(cudaStreamSynchronize(s));
                }
            } else if (!conv) {
                apply_one(h, h->d_r, h->d_z);
                dot_h(h, h->d_r, h->d_z, 4, tol2);
                ck(cudaMemcpyAsync(h->d_pv, h->d_z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                for (its = 1; its <= maxit; ++its) {
                    spmv_h(h, h->d_pv, h->d_q);
                    dot_h(h, h->d_pv, h->d_q, 0, tol2);
                    {
                        PScope ps(h, PK_PCG_VEC, 6.0 * n, 48.0 * n);
                        launch_pcg_update_xr(n, xk, h->d_r, h->d_pv, h->d_q, h->d_sc, h->d_part, s);
                    }
                    {
                        PScope ps(h, PK_PCG_VEC);
                        launch_dot_finalize(h->d_part, h->d_sc, 2, tol2, s);
                    }
                    ck(cudaMemcpyAsync(&sc, h->d_sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
                    ck(cudaStreamSynchronize(s));
                    if (k == 0) {
                        if (its > 1) be.push_back(sc.beta);
                        al.push_back(sc.alpha);
                    }
                    if (sc.conv) {
                        conv = true;
                        break;
                    }
                    if (its == maxit) break;
                    apply_one(h, h->d_r, h->d_z);
                    dot_h(h, h->d_r, h->d_z, 1, tol2);
                    PScope ps(h, PK_PCG_VEC, 2.0 * n, 24.0 * n);
                    launch_pcg_update_p(n, h->d_pv, h->d_z, h->d_sc, s);
                }
                if (its > maxit) its = maxit;
            }
            if (!conv) result = AMDD_ERR_NOCONV;
            if (k == 0 && stats) {
                // true residual b - A x
                spmv_h(h, xk, h->d_q);
                launch_axpby(n, 1.0, bk, -1.0, h->d_q, h->d_z, s);
                dot_h(h, h->d_z, h->d_z, 5, tol2);
                PcgScal st{};
                ck(cudaMemcpyAsync(&st, h->d_sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s));
                ck(cudaStreamSynchronize(s));
                stats->iterations = its;
                stats->converged = conv ? 1 : 0;
                stats->rel_residual = sc.bb > 0.0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
                stats->true_rel_residual = sc.bb > 0.0 ? std::sqrt(st.rr / sc.bb) : 0.0;
                lanczos_extremes(al, be, &stats->ritz_min, &stats->ritz_max);
                stats->cond_est = stats->ritz_max / stats->ritz_min;
            }
        }
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(s));
    } catch (...) {
        return guard_exc();
    }
    if (stats)
        stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return result;
}

amdd_status amdd_apply_form(amdd_handle* h, int32_t form, const double* r, double* z, int32_t nrhs) {
    if (!h || !r || !z || nrhs < 0 || r == z || form < AMDD_FORM_ADDITIVE || form > AMDD_FORM_ASM)
        return AMDD_ERR_INVALID;
    if (form == AMDD_FORM_ADDITIVE) return amdd_apply(h, r, z, nrhs);
    try {
        for (int k = 0; k < nrhs; ++k) apply_form(h, form, r + (size_t)k * h->n, z + (size_t)k * h->n);
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(h->s));
    } catch (...) {
        return guard_exc();
    }
    return AMDD_OK;
}

amdd_status amdd_gmres_solve(amdd_handle* h, int32_t form, const double* b, double* x, int32_t nrhs,
                             int32_t restart, double rtol, int32_t maxit, amdd_stats* stats) {
    if (!h || !b || !x || nrhs < 0 || !(rtol >= 0.0) || maxit < 0 || restart < 1 || restart > AMDD_GMRES_MAX_RESTART ||
        form < AMDD_FORM_ADDITIVE || form > AMDD_FORM_ASM)
        return AMDD_ERR_INVALID;
    const auto t0 = std::chrono::steady_clock::now();
    amdd_status result = AMDD_OK;
    try {
        cudaStream_t s = h->s;
        const int64_t n = h->n;
        // a NaN or infinity in b or in the initial guess: AMDD_ERR_INVALID
        require(all_finite(h, b, (int64_t)nrhs * n) && all_finite(h, x, (int64_t)nrhs * n));
        for (int k = 0; k < nrhs; ++k) {
            const double* bk = b + (size_t)k * n;
            double* xk = x + (size_t)k * n;
            const GmResult g = gmres_run(h, form, bk, xk, restart, rtol, maxit);
            if (!g.conv) result = AMDD_ERR_NOCONV;
            if (k == 0 && stats) {
                // true residual b - A x
                launch_spmv_resid(n, h->rowptr, h->col, h->val, xk, bk, h->d_gm_wA, h->spmv_group, s);
                launch_dot_partials(n, h->d_gm_wA, h->d_gm_wA, h->d_gm_part, s);
                launch_gm_norm(h->d_gm_part, h->d_gm_st, 0, s);
                double rr = 0.0;
                ck(cudaMemcpyAsync(&rr, reinterpret_cast<const char*>(h->d_gm_st) + offsetof(GmState, bnorm2),
                                   sizeof(double), cudaMemcpyDeviceToHost, s));
                ck(cudaStreamSynchronize(s));
                stats->iterations = g.its;
                stats->converged = g.conv ? 1 : 0;
                stats->rel_residual = g.bnorm2 > 0.0 ? g.res : 0.0;
                stats->true_rel_residual = g.bnorm2 > 0.0 ? std::sqrt(rr / g.bnorm2) : 0.0;
                stats->ritz_min = stats->ritz_max = stats->cond_est = std::numeric_limits<double>::quiet_NaN();
            }
        }
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(s));
        const int e = read_err(h);
        if (e) throw Fail{err_status(e)};
    } catch (...) {
        return guard_exc();
    }
    if (stats)
        stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return result;
}

amdd_status amdd_setup_next_level(amdd_handle* h, const int32_t* groups, int32_t N2, int32_t overlap2,
                                  double tau2, const amdd_opts* opts2, int32_t inner_restart, double inner_rtol,
                                  int32_t inner_maxit) {
    if (!h || !groups || !h->d_E_val || h->nC < 1 || N2 < 1 || inner_restart < 1 ||
        inner_restart > AMDD_GMRES_MAX_RESTART || !(inner_rtol >= 0.0) || inner_maxit < 1)
        return AMDD_ERR_INVALID;
    std::vector<int32_t> part2(h->nC);
    std::vector<int64_t> cnt(N2, 0);
    for (int i = 0; i < h->N; ++i) {
        if (groups[i] < 0 || groups[i] >= N2) return AMDD_ERR_INVALID;
        for (int k = 0; k < h->p[i]; ++k) part2[h->coff[i] + k] = groups[i];
        cnt[groups[i]] += h->p[i];
    }
    for (int g = 0; g < N2; ++g)
        if (cnt[g] == 0) return AMDD_ERR_INVALID;
    amdd_handle* h2 = nullptr;
    int32_t* d_part2 = nullptr;
    try {
        ck(cudaMallocAsync(reinterpret_cast<void**>(&d_part2), h->nC * sizeof(int32_t), h->s));
        ck(cudaMemcpyAsync(d_part2, part2.data(), h->nC * sizeof(int32_t), cudaMemcpyHostToDevice, h->s));
        ck(cudaStreamSynchronize(h->s));
    } catch (...) {
        if (d_part2) cudaFreeAsync(d_part2, h->s);
        return guard_exc();
    }
    const amdd_csr E{h->nC, h->E_nnz, h->d_E_rowptr, h->d_E_col, h->d_E_val};
    const amdd_status st = amdd_setup(&E, d_part2, N2, overlap2, tau2, opts2, h->s, &h2);
    cudaFreeAsync(d_part2, h->s);
    cudaStreamSynchronize(h->s);
    if (st != AMDD_OK) return st;
    amdd_destroy(h->next);
    h->next = h2;
    h->in_restart = inner_restart;
    h->in_rtol = inner_rtol;
    h->in_maxit = inner_maxit;
    h->in_calls = h->in_its = 0;
    h->in_max = 0;
    // the next level holds its own copy of E
    for (void* p : {static_cast<void*>(h->d_E_rowptr), static_cast<void*>(h->d_E_col), static_cast<void*>(h->d_E_val)}) {
        cudaFreeAsync(p, h->s);
        h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
    }
    h->d_E_rowptr = nullptr;
    h->d_E_col = nullptr;
    h->d_E_val = nullptr;
    cudaStreamSynchronize(h->s);
    return AMDD_OK;
}

amdd_handle* amdd_next_level(const amdd_handle* h) { return h ? h->next : nullptr; }

amdd_status amdd_get_info(const amdd_handle* h, amdd_info* info) {
    if (!h || !info) return AMDD_ERR_INVALID;
    std::memset(info, 0, sizeof(*info));
    info->n = h->n;
    info->N = h->N;
    info->overlap = h->overlap;
    info->tau = h->tau;
    info->n_C = h->nC;
    info->sum_ni = h->sum_ni;
    info->sum_nti = h->sum_nt;
    info->max_ni = h->max_ni;
    info->max_nti = h->max_nt;
    info->sweeps_svd = h->sweeps_svd;
    info->sweeps_eig = h->sweeps_eig;
    info->setup_ms = h->setup_ms;
    info->rotations_svd = h->rot_svd;
    info->rotations_eig = h->rot_eig;
    info->sweeps_svd32 = h->sweeps_svd32;
    info->sweeps_eig32 = h->sweeps_eig32;
    info->precision = h->precision;
    info->eps = h->eps;
    info->n_partial = h->n_partial;
    info->lobpcg_subdomains = h->lob_subs;
    info->lobpcg_fallbacks = h->lob_fallbacks;
    info->lobpcg_iters_max = h->lob_max;
    info->lobpcg_iters_total = h->lob_total;
    info->robust_schur = h->n_robust;
    info->levels = 1;
    for (const amdd_handle* q = h->next; q; q = q->next) info->levels += 1;
    info->inner_iterations_max = h->in_max;
    info->inner_solves = h->in_calls;
    info->inner_iterations = h->in_its;
    info->n_tied = h->n_tied;
    info->n_below_one = h->n_below_one;
    for (int k = 0; k < 10; ++k) info->pair_stats[k] = h->pair_stats[k];
    info->device_bytes_peak = (int64_t)h->bytes_peak;
    info->graph_solves = h->graph_solves;
    info->sparse_local_nnz = h->sparse_local ? h->sl_nnz : 0;
    {
        std::lock_guard<std::mutex> lock(tile_tuner().mu);
        info->tuned_buckets = tile_tuner().measured;
    }
    return AMDD_OK;
}

amdd_status amdd_get_subdomain(const amdd_handle* h, int32_t i, int32_t* nI, int32_t* nG, int32_t* nD, int32_t* p) {
    if (!h || i < 0 || i >= h->N) return AMDD_ERR_INVALID;
    if (nI) *nI = h->nI[i];
    if (nG) *nG = h->nG[i];
    if (nD) *nD = h->nD[i];
    if (p) *p = h->p[i];
    return AMDD_OK;
}

amdd_status amdd_get_eigenvalues(const amdd_handle* h, int32_t i, double* lam, int32_t cap, int32_t* count) {
    if (!h || i < 0 || i >= h->N) return AMDD_ERR_INVALID;
    const int c = h->nI[i];
    if (count) *count = c;
    if (lam) {
        if (cap < c) return AMDD_ERR_INVALID;
        std::memcpy(lam, h->lam_h.data() + h->off_I[i], c * sizeof(double));
    }
    return AMDD_OK;
}

amdd_status amdd_get_singular_values(const amdd_handle* h, int32_t i, double* sigma, int32_t cap, int32_t* count) {
    if (!h || i < 0 || i >= h->N) return AMDD_ERR_INVALID;
    const int c = h->ni[i];
    if (count) *count = c;
    if (sigma) {
        if (cap < c) return AMDD_ERR_INVALID;
        std::memcpy(sigma, h->sigma_h.data() + h->off_om[i], c * sizeof(double));
    }
    return AMDD_OK;
}

amdd_status amdd_get_coarse_block(const amdd_handle* h, int32_t i, double* Zt, int64_t cap, int32_t* p,
                                  int32_t* nI) {
    if (!h || i < 0 || i >= h->N) return AMDD_ERR_INVALID;
    const int64_t cnt = (int64_t)h->p[i] * h->nI[i];
    if (p) *p = h->p[i];
    if (nI) *nI = h->nI[i];
    if (Zt && cnt > 0) {
        if (cap < cnt) return AMDD_ERR_INVALID;
        if (cudaMemcpyAsync(Zt, h->d_Zt + h->off_zt[i], cnt * sizeof(double), cudaMemcpyDeviceToHost, h->s) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->s) != cudaSuccess)
            return AMDD_ERR_CUDA;
    }
    return AMDD_OK;
}

amdd_status amdd_get_profile(amdd_handle* h, int32_t k, const char** name, int64_t* launches, double* ms,
                             double* flops, double* bytes) {
    if (!h || !h->prof.on || k < 0 || k >= PK_COUNT) return AMDD_ERR_INVALID;
    if (cudaStreamSynchronize(h->s) != cudaSuccess) return AMDD_ERR_CUDA;
    double t = 0.0;
    for (auto& e : h->prof.ev[k]) {
        float x = 0.0f;
        if (cudaEventElapsedTime(&x, e.first, e.second) != cudaSuccess) return AMDD_ERR_CUDA;
        t += x;
    }
    if (name) *name = kProfNames[k];
    if (launches) *launches = h->prof.launches[k];
    if (ms) *ms = t;
    if (flops) *flops = h->prof.flops[k];
    if (bytes) *bytes = h->prof.bytes[k];
    return AMDD_OK;
}

amdd_status amdd_reset_profile(amdd_handle* h) {
    if (!h || !h->prof.on) return AMDD_ERR_INVALID;
    if (cudaStreamSynchronize(h->s) != cudaSuccess) return AMDD_ERR_CUDA;
    h->prof.clear();
    return AMDD_OK;
}

void amdd_destroy(amdd_handle* h) {
    if (!h) return;
    amdd_destroy(h->next);
    if (h->s2) cudaStreamSynchronize(h->s2);
    if (h->s3) cudaStreamSynchronize(h->s3);
    if (h->s4) cudaStreamSynchronize(h->s4);
    cudaStreamSynchronize(h->s);
    for (cudaEvent_t e : {h->ev_panel, h->ev_far, h->ev_panel3, h->ev_far3, h->ev_spec_in, h->ev_spec_done})
        if (e) cudaEventDestroy(e);
    if (h->s2) cudaStreamDestroy(h->s2);
    if (h->s3) cudaStreamDestroy(h->s3);
    if (h->s4) cudaStreamDestroy(h->s4);
    h->prof.release();
    if (h->pg_exec) cudaGraphExecDestroy(h->pg_exec);
    if (h->pg_graph) cudaGraphDestroy(h->pg_graph);
    if (h->s_cap) cudaStreamDestroy(h->s_cap);
    for (void* p : h->allocs) cudaFreeAsync(p, h->s);
    cudaStreamSynchronize(h->s);
    delete h;
}

const char* amdd_status_str(amdd_status s) {
    switch (s) {
        case AMDD_OK: return "ok";
        case AMDD_ERR_INVALID: return "invalid argument";
        case AMDD_ERR_NOT_SPD: return "matrix not SPD (Cholesky pivot <= 0)";
        case AMDD_ERR_NOCONV: return "PCG did not converge within maxit";
        case AMDD_ERR_OOM: return "out of memory";
        case AMDD_ERR_TIMEOUT: return "device wait timed out";
        case AMDD_ERR_CUDA: return "CUDA runtime error";
        case AMDD_ERR_EIG_NOCONV: return "Jacobi eigensolver did not converge";
    }
    return "unknown status";
}

}  // extern "C"
