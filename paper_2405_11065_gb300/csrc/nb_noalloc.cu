// glsc3 without any allocation: the weighted dot product of nb_glsc3 with its
// scratch (the per-block partial sums and the final scalar) in a fixed
// device array instead of buffers obtained from cudaMalloc.
//
// Some callers cannot let a library allocate device or pinned memory: a
// framework whose caching allocator already owns all device memory, a
// process running under a hard memory budget where a late allocation could
// fail or fragment the heap, and latency-critical loops where cudaMalloc's
// implicit device-wide synchronisation is not acceptable.  nb_glsc3 allocates
// its scratch lazily on first use; this entry point never does.
#include <algorithm>

#include "nb_reduce.cuh"

namespace nb {

// Scratch shared by every call on a device: kNoAllocSlots partial sums and,
// in the last slot, the result.  Every slot a call reads is written earlier
// in the same call, so nothing has to be cleared between calls; the array
// keeps the previous call's values until overwritten.
constexpr int kNoAllocSlots = 2048;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots + 1];

// Device address of g_noalloc_scratch per device, looked up once with that
// device current (host code cannot use the symbol itself as an address).
constexpr int kNoAllocMaxDevices = 64;
static double *g_scratch_addr[kNoAllocMaxDevices] = {};

static nb_status noalloc_scratch(int device, double **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices) {
        set_error("device index %d beyond the no-allocation scratch table", device);
        return NB_ERR_ARG;
    }
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        NB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[device];
    return NB_OK;
}

template <typename T>
__global__ void k_glsc3_noalloc_part(int64_t n, const T *__restrict__ a, const T *__restrict__ b,
                                     const float *__restrict__ c, double *__restrict__ part)
{
    __shared__ double sred[32];
    double acc = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        acc += (double)(a[l] * b[l] * (T)c[l]);
    double t = block_sum(acc, sred);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_glsc3_noalloc_final(const double *__restrict__ part, int cnt,
                                      double *__restrict__ out)
{
    __shared__ double sred[32];
    double t = sum_partials(part, cnt, sred);
    if (threadIdx.x == 0) *out = t;
}

}  // namespace nb

using namespace nb;

extern "C" nb_status nb_glsc3_noalloc(nb_mesh *m, nb_prec prec, const void *a, const void *b,
                                      double *out_host)
{
    if (!m || !a || !b || !out_host) {
        set_error("invalid argument: NULL mesh, vector or output");
        return NB_ERR_ARG;
    }
    if (prec < NB_FP64 || prec > NB_TC_BF16) {
        set_error("invalid argument: precision");
        return NB_ERR_ARG;
    }
    if (!m->gs_ready) {
        set_error("call nb_setup_gs first");
        return NB_ERR_STATE;
    }
    NB_DEVICE_SCOPE(m->ctx->device);
    const int grid = vec_grid(m->ctx, m->nL);
    if (grid > kNoAllocSlots) {
        set_error("nb_glsc3_noalloc: %d partial sums exceed the fixed scratch of %d", grid,
                  kNoAllocSlots);
        return NB_ERR_ARG;
    }
    double *scratch = nullptr;
    NB_TRY(noalloc_scratch(m->ctx->device, &scratch));
    cudaStream_t s = m->ctx->stream;
    if (prec == NB_FP64)
        k_glsc3_noalloc_part<double><<<grid, kVecThreads, 0, s>>>(
            m->nL, (const double *)a, (const double *)b, m->c32, scratch);
    else
        k_glsc3_noalloc_part<float><<<grid, kVecThreads, 0, s>>>(
            m->nL, (const float *)a, (const float *)b, m->c32, scratch);
    NB_CUDA(cudaGetLastError());
    k_glsc3_noalloc_final<<<1, kFinalizeThreads, 0, s>>>(scratch, grid, scratch + kNoAllocSlots);
    NB_CUDA(cudaGetLastError());
    NB_CUDA(cudaMemcpyAsync(out_host, scratch + kNoAllocSlots, sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    NB_CUDA(cudaStreamSynchronize(s));
    return NB_OK;
}
