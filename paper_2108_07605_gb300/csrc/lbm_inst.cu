// One instantiation of the kernel templates, selected on the compiler
// command line: LBM_D (2 or 3), LBM_M (species), LBM_F64 (1: FP64 storage
// and arithmetic; 0: FP32 storage, mixed arithmetic) and LBM_KSET (the
// accessor's name).  Each combination is its own translation unit so that
// the build compiles them in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

#if LBM_F64
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, double, double>(); }
#else
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, float, float>(); }
#endif

}  // namespace lbm
