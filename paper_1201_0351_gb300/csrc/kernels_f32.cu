// Kernels of the free-surface LBM step for one population storage (see
// lbmfs_kernels.cuh).
#include "lbmfs_kernels.cuh"

namespace lbmfs {
KernelSet kernels_f32() { return make_kernel_set<1>(); }
}  // namespace lbmfs
