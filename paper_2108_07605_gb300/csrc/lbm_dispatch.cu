// Dispatch from (lattice, species count, precision) to the kernel sets
// instantiated by lbm_inst.cu, plus the precision-only conversion kernel.
#include <algorithm>

#include "lbm_internal.h"

namespace lbm {

const KernelSet* kernel_set_3_9_f64();
const KernelSet* kernel_set_3_9_f32();
const KernelSet* kernel_set_3_2_f64();
const KernelSet* kernel_set_3_2_f32();
const KernelSet* kernel_set_2_9_f64();
const KernelSet* kernel_set_2_9_f32();
const KernelSet* kernel_set_2_2_f64();
const KernelSet* kernel_set_2_2_f32();

const KernelSet* kernel_set(int D, int M, lbm_precision prec) {
  const bool f64 = prec == LBM_FP64;
  if (prec != LBM_FP64 && prec != LBM_FP32_STORE) return nullptr;
  if (D == 3 && M == 9) return f64 ? kernel_set_3_9_f64() : kernel_set_3_9_f32();
  if (D == 3 && M == 2) return f64 ? kernel_set_3_2_f64() : kernel_set_3_2_f32();
  if (D == 2 && M == 9) return f64 ? kernel_set_2_9_f64() : kernel_set_2_9_f32();
  if (D == 2 && M == 2) return f64 ? kernel_set_2_2_f64() : kernel_set_2_2_f32();
  return nullptr;
}

cudaError_t launch_step(int D, int M, lbm_precision prec, const DevMech& mech,
                        const StepArgs& a, cudaStream_t s, int which) {
  const KernelSet* k = kernel_set(D, M, prec);
  return k ? k->step(mech, a, s, which) : cudaErrorInvalidValue;
}

cudaError_t launch_init(int D, int M, lbm_precision prec, const DevMech& mech,
                        const Geom& g, const Units& un, const double* rho_or_P,
                        int is_pressure, const double* u, const double* T,
                        const double* Y, void* pops, double* Tfield, int* status,
                        cudaStream_t s) {
  const KernelSet* k = kernel_set(D, M, prec);
  return k ? k->init(mech, g, un, rho_or_P, is_pressure, u, T, Y, pops, Tfield, status, s)
           : cudaErrorInvalidValue;
}

cudaError_t launch_moments_out(int D, int M, lbm_precision prec, const DevMech& mech,
                               const Geom& g, const Units& un, const void* pops,
                               const double* Tfield, double* rho, double* u, double* T,
                               double* Y, double* E, int* status, cudaStream_t s) {
  const KernelSet* k = kernel_set(D, M, prec);
  return k ? k->out(mech, g, un, pops, Tfield, rho, u, T, Y, E, status, s)
           : cudaErrorInvalidValue;
}

cudaError_t prepare_batch_step(int D, int M, lbm_precision prec) {
  const KernelSet* k = kernel_set(D, M, prec);
  return k ? k->prepare() : cudaErrorInvalidValue;
}

cudaError_t launch_batch_step(int D, int M, lbm_precision prec, const DomainDev* doms,
                              int ndom, const BatchGrids& gr, const Launch& lc, int parity,
                              cudaStream_t s, const SideStream& side) {
  const KernelSet* k = kernel_set(D, M, prec);
  return k ? k->batch(doms, ndom, gr, lc, parity, s, side) : cudaErrorInvalidValue;
}

int record_fields(int D, int M) {
  const KernelSet* k = kernel_set(D, M, LBM_FP64);
  return k ? k->record_fields : -1;
}

int collide_param_fields(int D, int M) {
  const KernelSet* k = kernel_set(D, M, LBM_FP64);
  return k ? k->param_fields : -1;
}

// populations of either storage type as FP64
template <typename S>
__global__ void k_to_fp64(const S* __restrict__ in, double* __restrict__ out, long long count) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = static_cast<double>(in[k]);
}

cudaError_t launch_to_fp64(lbm_precision prec, const void* pops, double* out,
                           long long count, cudaStream_t s) {
  const long long nb = std::min<long long>((count + 255) / 256, 152LL * 16);
  if (nb <= 0) return cudaSuccess;
  if (prec == LBM_FP64)
    k_to_fp64<double><<<(unsigned)nb, 256, 0, s>>>(static_cast<const double*>(pops), out, count);
  else if (prec == LBM_FP32_STORE)
    k_to_fp64<float><<<(unsigned)nb, 256, 0, s>>>(static_cast<const float*>(pops), out, count);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lbm
