// lbm_fs_liquid_mass_noalloc: the liquid-mass reduction with its block
// partial sums in a fixed device array instead of library-allocated scratch.
//
// For callers that must not allocate device memory: an application that
// hands the library a fixed memory budget and owns every allocation, code that
// runs while a CUDA graph is being captured (an allocation would end the
// capture), or a latency-critical loop where a cudaMalloc / cudaFree could
// block on device synchronisation.  The caller passes device pointers to the
// inputs and the output; nothing is allocated.
#include <cuda.h>  // CUcontext / CUresult types of the two driver calls looked up below
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "lbm_fs.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 4096;      // cells summed by one block
constexpr int NA_SCRATCH = 65536;         // block partial sums held (512 KiB)
constexpr int NA_MAX_DEVICES = 64;

// Shared by every call on a device; keeps the last call's partial sums.
static __device__ __align__(256) double g_mass_partials[NA_SCRATCH];

// device address of the array per device, with the id of the context it was
// looked up in: a cudaDeviceReset, or a caller's own (non-primary) context,
// brings a new context in which the library's device code, and the array,
// may sit elsewhere, so the address is looked up again for a new context id
struct Setup {
    unsigned long long ctx_id;
    double *ptr;
};
Setup g_setup[NA_MAX_DEVICES];
std::mutex g_setup_mutex;
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// id of the calling thread's current context (0 on failure); call with
// g_setup_mutex held
unsigned long long current_context_id(int dev) {
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&g_ctx_current, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&g_ctx_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            g_ctx_current = nullptr;
            g_ctx_id = nullptr;
            return 0;
        }
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return 0;
    if (!ctx) {
        // no context yet on this thread: make the device's primary context current
        if (cudaSetDevice(dev) != cudaSuccess || g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    }
    unsigned long long id = 0;
    return g_ctx_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}
thread_local std::string g_na_err;

__global__ void k_na_partial(const uint8_t *flags, const double *mass, long long n, double *partials) {
    long long base = blockIdx.x * NA_CHUNK;
    long long end = base + NA_CHUNK < n ? base + NA_CHUNK : n;
    double acc = 0.0;
    for (long long i = base + threadIdx.x; i < end; i += blockDim.x) {
        int c = flags[i] & 15;
        if (c == LBM_FS_LIQUID || c == LBM_FS_INTERFACE) acc += mass[i];
    }
    __shared__ double sh[NA_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
        partials[blockIdx.x] = t;  // every block overwrites its slot: no clearing needed
    }
}

__global__ void k_na_final(const double *partials, int nblocks, double *out) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) acc += partials[k];
    __shared__ double sh[NA_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) t += sh[w];
        *out = t;
    }
}

lbm_fs_status na_fail(lbm_fs_status s, const char *msg) {
    g_na_err = msg;
    return s;
}

}  // namespace

extern "C" lbm_fs_status lbm_fs_liquid_mass_noalloc(const uint8_t *flags, const double *mass, int64_t n,
                                                   double *out, void *stream) {
    if (!flags || !mass || !out) return na_fail(LBM_FS_EINVAL, "lbm_fs_liquid_mass_noalloc: null pointer");
    if (n < 0 || n > (int64_t)NA_CHUNK * NA_SCRATCH)
        return na_fail(LBM_FS_EINVAL,
                       "lbm_fs_liquid_mass_noalloc: n must lie in [0, 268435456] (the fixed partial-sum array "
                       "holds 65536 blocks of 4096 cells)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(LBM_FS_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(LBM_FS_EINVAL, "lbm_fs_liquid_mass_noalloc: device index");
    double *partials;
    {
        // set-up, once per device and context, with that device current: the
        // host-side name of the array is not a device address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        const unsigned long long id = current_context_id(dev);
        if (id == 0) return na_fail(LBM_FS_ECUDA, "lbm_fs_liquid_mass_noalloc: no current CUDA context");
        if (!g_setup[dev].ptr || g_setup[dev].ctx_id != id) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_mass_partials);
            if (e != cudaSuccess) return na_fail(LBM_FS_ECUDA, cudaGetErrorString(e));
            g_setup[dev].ptr = (double *)ptr;
            g_setup[dev].ctx_id = id;
        }
        partials = g_setup[dev].ptr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int nblocks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    if (nblocks > 0) k_na_partial<<<nblocks, NA_THREADS, 0, st>>>(flags, mass, (long long)n, partials);
    k_na_final<<<1, NA_THREADS, 0, st>>>(partials, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(LBM_FS_ECUDA, cudaGetErrorString(e));
    return LBM_FS_OK;
}

extern "C" const char *lbm_fs_noalloc_last_error_string(void) { return g_na_err.c_str(); }
