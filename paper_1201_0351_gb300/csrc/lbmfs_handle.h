// The simulation handle behind the C ABI and the host helpers shared by the
// single-tank API and the batched form (private to the library).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "lbm_fs.h"
#include "lbmfs_internal.h"

struct lbm_fs {
    lbm_fs_params p;
    lbmfs::KernelSet ks;
    lbmfs::Dev d[2];  // d[0] streams A -> B, d[1] streams B -> A
    int cur = 0;
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    std::vector<void *> allocs;
    int nb = 0;
    bool started = false;
    int64_t step = 0;
    int64_t launches = 0;
    int per_step = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_nb = -1;
    bool dead = false;
    lbm_fs_batch *owner = nullptr;  // set while the tank belongs to a batch
    bool misaligned = false;        // a dev_alloc result was not 16-byte aligned

    void *alloc(size_t bytes) {
        void *ptr = nullptr;
        if (bytes == 0) bytes = 4;
        if (p.dev_alloc) {
            ptr = p.dev_alloc(bytes, p.alloc_ctx);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
        if (ptr) allocs.push_back(ptr);
        if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 15u)) misaligned = true;  // vector loads need 16 bytes
        return ptr;
    }
    void release() {
        for (int k = 0; k < 2; ++k)
            if (gexec[k]) cudaGraphExecDestroy(gexec[k]);
        for (void *ptr : allocs) {
            if (p.dev_free) p.dev_free(ptr, p.alloc_ctx);
            else cudaFree(ptr);
        }
        allocs.clear();
        if (cap_st) cudaStreamDestroy(cap_st);
    }
};

namespace lbmfs {
// record the failure text of the calling thread and return the status
lbm_fs_status fail(lbm_fs_status s, const char *fmt, const char *detail = nullptr);
lbm_fs_status cuda_fail(cudaError_t e, const char *where);
lbm_fs_status check_handle(lbm_fs *h);
// synchronise the handle's stream and map its sticky device bits to a status
lbm_fs_status read_status(lbm_fs *h);
// map a copy of the device status word to a status (first sticky bit wins)
lbm_fs_status status_bits(uint32_t st);
// before the first step: book the initial liquid mass (enqueued on h->st)
void begin_mass(lbm_fs *h);
}  // namespace lbmfs

#define LBMFS_CK(call)                                                 \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::lbmfs::cuda_fail(e_, #call);   \
    } while (0)
