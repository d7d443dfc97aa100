// Measurement helper: the double-precision instruction rate of this GPU,
// against which the double-storage path (bound by double arithmetic, not by
// memory) is quoted.  Independent chains of one FP64 operation per thread,
// enough resident warps to fill every SM, timed with CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_fs.h"

namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_CHAINS = 8;  // independent dependency chains per thread

// written only when the chains end on an impossible value: keeps the
// arithmetic alive without a result buffer to allocate
__device__ double g_probe_sink;

template <int OP>
__global__ void __launch_bounds__(PR_THREADS) k_fp64_rate(int iters, double a, double b) {
    double x[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < PR_CHAINS; ++c) {
            if (OP == 0) x[c] = __fma_rn(x[c], a, b);
            else if (OP == 1) x[c] = __dadd_rn(x[c], b);
            else x[c] = __dmul_rn(x[c], a);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
    if (s == -1.2345678e300) g_probe_sink = s;
}

}  // namespace

extern "C" lbm_fs_status lbm_fs_fp64_rate(int32_t op, int32_t iters, double *ops_per_s, void *stream) {
    if (!ops_per_s || op < 0 || op > 2 || iters <= 0) return LBM_FS_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_FS_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    switch (op) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate<0>, PR_THREADS, 0); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate<1>, PR_THREADS, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate<2>, PR_THREADS, 0); break;
    }
    if (e != cudaSuccess || per_sm <= 0) return LBM_FS_ECUDA;
    const int blocks = sms * per_sm;
    // values that stay finite and normal over any number of iterations
    const double a = 0.9999999, b = 1e-9;
    auto launch = [&](int n) {
        switch (op) {
            case 0: k_fp64_rate<0><<<blocks, PR_THREADS, 0, st>>>(n, a, b); break;
            case 1: k_fp64_rate<1><<<blocks, PR_THREADS, 0, st>>>(n, a, b); break;
            default: k_fp64_rate<2><<<blocks, PR_THREADS, 0, st>>>(n, a, b); break;
        }
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_FS_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBM_FS_ECUDA;
    }
    launch(iters / 10 + 1);  // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0.0f) return LBM_FS_ECUDA;
    *ops_per_s = (double)blocks * PR_THREADS * PR_CHAINS * (double)iters / (ms * 1e-3);
    return LBM_FS_OK;
}
