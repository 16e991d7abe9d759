// Dispatch from (lattice, species count, precision) to the kernel sets
// instantiated by lbm_inst.cu, plus the precision-only conversion kernel.
#include <algorithm>
#include <climits>

#include "lbm_internal.h"

namespace lbm {

#define LBM_DECLARE_SETS(D_, M_)                 \
  const KernelSet* kernel_set_##D_##_##M_##_f64(); \
  const KernelSet* kernel_set_##D_##_##M_##_f32(); \
  const KernelSet* kernel_set_##D_##_##M_##_c64(); \
  const KernelSet* kernel_set_##D_##_##M_##_f16();
LBM_DECLARE_SETS(3, 9)
LBM_DECLARE_SETS(3, 2)
LBM_DECLARE_SETS(2, 9)
LBM_DECLARE_SETS(2, 2)
#undef LBM_DECLARE_SETS

const KernelSet* kernel_set(int D, int M, lbm_precision prec) {
#define LBM_PICK(D_, M_)                                                      \
  if (D == D_ && M == M_) {                                                   \
    if (prec == LBM_FP64) return kernel_set_##D_##_##M_##_f64();              \
    if (prec == LBM_FP32_STORE) return kernel_set_##D_##_##M_##_f32();        \
    if ((int)prec == LBM_KPREC_FP32_CHEM64) return kernel_set_##D_##_##M_##_c64(); \
    if (prec == LBM_FP16_OFFSET) return kernel_set_##D_##_##M_##_f16();       \
    return nullptr;                                                           \
  }
  LBM_PICK(3, 9)
  LBM_PICK(3, 2)
  LBM_PICK(2, 9)
  LBM_PICK(2, 2)
#undef LBM_PICK
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

// the per-block partials of k_diag reduced in a fixed order by one block
__global__ void k_diag_final(const DiagPart* __restrict__ part, int nb, DiagPart* out) {
  __shared__ DiagPart s[256];
  const int t = threadIdx.x;
  DiagPart a{0.0, -INFINITY, LLONG_MAX, -INFINITY, -INFINITY};
  for (int b = t; b < nb; b += blockDim.x) {
    const DiagPart p = part[b];
    a.q_sum += p.q_sum;
    if (p.q_max > a.q_max || (p.q_max == a.q_max && p.n_max < a.n_max)) {
      a.q_max = p.q_max;
      a.n_max = p.n_max;
    }
    a.T_max = fmax(a.T_max, p.T_max);
    a.u_max = fmax(a.u_max, p.u_max);
  }
  s[t] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) {
      DiagPart& x = s[t];
      const DiagPart& y = s[t + o];
      x.q_sum += y.q_sum;
      if (y.q_max > x.q_max || (y.q_max == x.q_max && y.n_max < x.n_max)) {
        x.q_max = y.q_max;
        x.n_max = y.n_max;
      }
      x.T_max = fmax(x.T_max, y.T_max);
      x.u_max = fmax(x.u_max, y.u_max);
    }
    __syncthreads();
  }
  if (t == 0) *out = s[0];
}

cudaError_t launch_diagnostics(int D, int M, lbm_precision prec, const DevMech& mech,
                               const Geom& g, const Units& un, const void* pops,
                               const double* Tfield, const int* tag, DiagPart* part,
                               DiagPart* out, int* status, int x0, int x1, cudaStream_t s) {
  const KernelSet* k = kernel_set(D, M, prec);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = k->diag(mech, g, un, pops, Tfield, tag, part, status, x0, x1, s);
  if (e != cudaSuccess) return e;
  const int nb = (int)((g.N + 127) / 128);
  k_diag_final<<<1, 256, 0, s>>>(part, nb, out);
  return cudaGetLastError();
}

int record_fields(int D, int M) {
  const KernelSet* k = kernel_set(D, M, LBM_FP64);
  return k ? k->record_fields : -1;
}

int collide_param_fields(int D, int M) {
  const KernelSet* k = kernel_set(D, M, LBM_FP64);
  return k ? k->param_fields : -1;
}

// populations of any storage type as FP64 (FP16: decoded, population index
// k / N of the layout [l*Q + i][N])
template <typename S>
__global__ void k_to_fp64(const S* __restrict__ in, double* __restrict__ out, long long count,
                          long long N, const float4* __restrict__ codec) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(S) == 2) {
      const float4 c = __ldg(codec + k / N);
      out[k] = (double)fmaf(c.y, __half2float(in[k]), c.x);
    } else {
      out[k] = static_cast<double>(in[k]);
    }
  }
}

cudaError_t launch_to_fp64(lbm_precision prec, const void* pops, double* out,
                           long long count, cudaStream_t s, long long N, const float4* codec) {
  const long long nb = std::min<long long>((count + 255) / 256, 152LL * 16);
  if (nb <= 0) return cudaSuccess;
  if (prec == LBM_FP64)
    k_to_fp64<double><<<(unsigned)nb, 256, 0, s>>>(static_cast<const double*>(pops), out, count,
                                                   N, codec);
  else if (prec == LBM_FP32_STORE)
    k_to_fp64<float><<<(unsigned)nb, 256, 0, s>>>(static_cast<const float*>(pops), out, count,
                                                  N, codec);
  else if (prec == LBM_FP16_OFFSET && codec)
    k_to_fp64<__half><<<(unsigned)nb, 256, 0, s>>>(static_cast<const __half*>(pops), out,
                                                   count, N, codec);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Codec of FP16 storage from FP32 equilibrium populations eq [L*Q][N] of the
// initial fields and the populations off [L*Q] of their mean state: per
// lattice the largest |eq - off| and the largest |eq| (as the bit patterns of
// non-negative floats, whose order is that of the values).
__global__ void k_codec_extent(const float* __restrict__ eq, const float* __restrict__ off,
                               int L, int Q, long long N, unsigned* __restrict__ dev_max,
                               unsigned* __restrict__ abs_max) {
  const int l = blockIdx.y;
  unsigned md = 0u, ma = 0u;
  for (int i = 0; i < Q; ++i) {
    const float o = off[l * Q + i];
    const float* row = eq + (long long)(l * Q + i) * N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
      const float v = row[n];
      md = max(md, __float_as_uint(fabsf(v - o)));
      ma = max(ma, __float_as_uint(fabsf(v)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
    ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(dev_max + l, md);
    atomicMax(abs_max + l, ma);
  }
}

// FP32 populations to FP16 offsets with the codec
__global__ void k_codec_encode(const float* __restrict__ eq, __half* __restrict__ out,
                               long long count, long long N,
                               const float4* __restrict__ codec) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const float4 c = __ldg(codec + k / N);
    out[k] = __float2half_rn((eq[k] - c.x) * c.z);
  }
}

cudaError_t launch_codec_extent(const float* eq, const float* off, int L, int Q, long long N,
                                unsigned* dev_max, unsigned* abs_max, cudaStream_t s) {
  const long long bx = std::min<long long>((N + 255) / 256, 64);
  k_codec_extent<<<dim3((unsigned)std::max<long long>(bx, 1), L), 256, 0, s>>>(
      eq, off, L, Q, N, dev_max, abs_max);
  return cudaGetLastError();
}

cudaError_t launch_codec_encode(const float* eq, void* out, long long count, long long N,
                                const float4* codec, cudaStream_t s) {
  const long long nb = std::min<long long>((count + 255) / 256, 152LL * 16);
  if (nb <= 0) return cudaSuccess;
  k_codec_encode<<<(unsigned)nb, 256, 0, s>>>(eq, static_cast<__half*>(out), count, N, codec);
  return cudaGetLastError();
}

}  // namespace lbm
