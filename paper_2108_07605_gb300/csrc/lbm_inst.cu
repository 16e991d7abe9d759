// One instantiation of the kernel templates, selected on the compiler
// command line: LBM_D (2 or 3), LBM_M (species), LBM_PREC (0: FP64 storage
// and arithmetic; 1: FP32 storage, mixed arithmetic; 2: FP16 offset
// storage, the FP32 path's arithmetic; 3: FP32 storage and lattice
// arithmetic with the temperature solve and chemistry in native FP64, built
// with LBM_CHEM64 = 1) and LBM_KSET (the accessor's name).
// Each combination is its own translation unit so that the build compiles
// them in parallel.
#include "lbm_kernels.cuh"

namespace lbm {

#if LBM_PREC == 0
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, double, double>(); }
#elif LBM_PREC == 1 || LBM_PREC == 3
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, float, float>(); }
#else
const KernelSet* LBM_KSET() { return make_kernel_set<LBM_D, LBM_M, __half, float>(); }
#endif

}  // namespace lbm
