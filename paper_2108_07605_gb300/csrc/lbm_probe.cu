// Measured FMA throughput of the GPU, the ALU roof that the step's executed
// FP32 / FP64 operation counts are compared against.  No counterpart in the
// paper: a measurement probe.
//
// Every thread runs eight independent fused multiply-add chains
// x <- x a + b (a = 0.999, b = 1e-3 keep x bounded), so the pipes are never
// short of independent work; the grid holds eight 256-thread blocks per SM.
// FLOP = 2 per FMA.  The kernel is timed with CUDA events, the best of three
// launches after a warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "lbm_internal.h"
#include "lbm_sync.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, int iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == T(-1.25)) out[0] = s;        // never true; keeps the chains live
}

template <typename T>
cudaError_t time_fma(int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  const int blocks = 8 * sms, threads = 256;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(t0);
    k_fma_peak<T><<<blocks, threads>>>(T(0.999), T(1e-3), iters, out);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * 8.0 * iters * (double)blocks * threads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return cudaSuccess;
}

// One thread waits on words[0] (abort word words[1]) with the persistent
// step's bounded wait; out[0] = 1 if the wait saw the word set, out[1] = the
// abort word afterwards, out[2] = the wait's length in microseconds.
__global__ void k_wait_probe(int* words, long long timeout_ns, long long* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long t0 = lbm::global_ns();
  const bool ok = lbm::wait_at_least(words, 1, words + 1, timeout_ns);
  out[0] = ok ? 1 : 0;
  out[1] = lbm::ld_acquire_gpu(words + 1);
  out[2] = (long long)((lbm::global_ns() - t0) / 1000ull);
}

}  // namespace

extern "C" lbm_status lbm_wait_probe(int set_word, long long timeout_ns, long long* result) {
  if (!result || timeout_ns < 0) return LBM_ERR_INVALID;
  if (timeout_ns > 100000000LL) return LBM_ERR_RANGE;
  int* words = nullptr;
  long long* out = nullptr;
  cudaError_t e = cudaMalloc(&words, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&out, 3 * sizeof(long long));
  const int init[2] = {set_word ? 1 : 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(words, init, sizeof(init), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_wait_probe<<<1, 32>>>(words, timeout_ns, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(result, out, 3 * sizeof(long long), cudaMemcpyDeviceToHost);
  if (words) cudaFree(words);
  if (out) cudaFree(out);
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

extern "C" lbm_status lbm_fma_peak(int fp64, double* tflops) {
  if (!tflops) return LBM_ERR_INVALID;
  const cudaError_t e = fp64 ? time_fma<double>(512, tflops) : time_fma<float>(16384, tflops);
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
