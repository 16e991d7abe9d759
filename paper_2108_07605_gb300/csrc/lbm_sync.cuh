// Device-wide release / acquire on sync words and a bounded wait on them
// (the persistent step's dependencies).  No counterpart in the paper.
#pragma once

namespace lbm {

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void add_release_gpu(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until *word >= want; false if the abort word is set or the wait
// outlasts timeout_ns (which then sets it).
__device__ __forceinline__ bool wait_at_least(const int* word, int want, int* abort_w,
                                              long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  unsigned sleep = 32;
  for (;;) {
    if (ld_acquire_gpu(word) >= want) return true;
    if (ld_acquire_gpu(abort_w)) return false;
    if ((long long)(global_ns() - t0) > timeout_ns) {
      atomicExch(abort_w, 1);
      return false;
    }
    __nanosleep(sleep);
    if (sleep < 2048) sleep *= 2;
  }
}

}  // namespace lbm
