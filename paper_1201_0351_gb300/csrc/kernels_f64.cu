// FP64 kernel set (compiled with -fmad=false: every operation rounded as the
// plain CPU restatement of the method rounds it), and the rigid-body update
// that every storage's kernel set launches.
#include "lbmfs_kernels.cuh"

namespace lbmfs {
KernelSet kernels_f64() { return make_kernel_set<0>(); }

void launch_bodies(const Dev &d, cudaStream_t st) { k_bodies<<<d.nb, 32, 0, st>>>(d); }
void launch_bodies_batch(const BatchLaunch &b, cudaStream_t st) { batch_launch<BkBodies>(b, SH_BODY, 32, st); }
}  // namespace lbmfs
