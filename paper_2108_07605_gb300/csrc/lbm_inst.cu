// One instantiation of the kernel templates, selected on the compiler
// command line: LBM_D (2 or 3), LBM_M (species), LBM_PREC (0: FP64 storage
// and arithmetic; 1: FP32 storage, mixed arithmetic; 2: FP16 offset
// storage, the FP32 path's arithmetic) and LBM_KSET (the accessor's name).
// Each combination is its own translation unit so that the build compiles
// them in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

#if LBM_PREC == 0
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, double, double>(); }
#elif LBM_PREC == 1
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, float, float>(); }
#else
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, __half, float>(); }
#endif

}  // namespace lbm
