// Entry point for callers that cannot allocate device memory: the true
// relative residual ||b - A x||_2 / ||b||_2 computed with the same kernels
// and the same fixed reduction order as amdd_pcg_solve's exit check, with all
// scratch in a file-scope device array instead of memory from cudaMalloc.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "amdd.h"
#include "amdd_internal.h"

using namespace amdd;

namespace {

// Scratch layout: A x and b - A x (AMDD_NOALLOC_MAX_N doubles each), the
// DOT_BLOCKS partial sums, then one PcgScal record.
constexpr size_t kScalDoubles = (sizeof(PcgScal) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kScratchDoubles = 2 * (size_t)AMDD_NOALLOC_MAX_N + DOT_BLOCKS + kScalDoubles;

static __device__ __align__(256) double g_residual_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name in host code is only a host-side stand-in).
amdd_status scratch_on_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMDD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_residual_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return AMDD_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return AMDD_OK;
}

}  // namespace

extern "C" amdd_status amdd_true_residual_noalloc(const amdd_csr* A, const double* b, const double* x, double* out,
                                                  void* stream) {
    if (!A || !b || !x || !out || A->n < 1 || A->nnz < 0 || !A->rowptr || (A->nnz > 0 && (!A->colind || !A->val)))
        return AMDD_ERR_INVALID;
    if (A->n > (int64_t)AMDD_NOALLOC_MAX_N) return AMDD_ERR_INVALID;  // larger than the static scratch
    double* scratch = nullptr;
    const amdd_status st = scratch_on_current_device(&scratch);
    if (st != AMDD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* q = scratch;
    double* r = scratch + AMDD_NOALLOC_MAX_N;
    double* partials = scratch + 2 * (size_t)AMDD_NOALLOC_MAX_N;
    PcgScal* sc = reinterpret_cast<PcgScal*>(partials + DOT_BLOCKS);
    const int64_t n = A->n;
    // the record keeps the previous call's values: clear it
    if (cudaMemsetAsync(sc, 0, sizeof(PcgScal), s) != cudaSuccess) return AMDD_ERR_CUDA;
    launch_spmv(n, A->rowptr, A->colind, A->val, x, q, spmv_group_for(n, A->nnz), s);
    launch_axpby(n, 1.0, b, -1.0, q, r, s);
    launch_dot_partials(n, b, b, partials, s);
    launch_dot_finalize(partials, sc, 3, 0.0, s);
    launch_dot_partials(n, r, r, partials, s);
    launch_dot_finalize(partials, sc, 5, 0.0, s);
    PcgScal h{};
    if (cudaMemcpyAsync(&h, sc, sizeof(PcgScal), cudaMemcpyDeviceToHost, s) != cudaSuccess) return AMDD_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return AMDD_ERR_CUDA;
    out[0] = std::sqrt(h.rr);
    out[1] = std::sqrt(h.bb);
    return AMDD_OK;
}
