// Space-time snapshot gather shared by the covariance and apply kernels.
//   x_{k,r}[t*C + c] = dop[c][(k + t - floor(T/2)) mod K][r]
// The snapshot tensor is never materialised in HBM: each CTA stages the
// D x ncells tile it needs into shared memory, row d = t*C + c contiguous in
// range, with leading dimension ld (padded so that reads of different rows at
// the same cell fall in different banks).
#pragma once

#include <mutex>

#include "stap_internal.cuh"

namespace stap {

__device__ __forceinline__ void stage_snapshots(float2* __restrict__ xs, int ld,
                                                const float2* __restrict__ dop, int C, int K, int ldr,
                                                int T, int k, int r_begin, int ncells) {
  // one warp per snapshot row, lanes along range: coalesced, no divisions per element
  const int D = C * T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < D; d += nw) {
    const int t = d / C, c = d - t * C;
    const int kk = wrap_bin(k + t - T / 2, K);
    const float2* src = dop + ((size_t)c * K + kk) * ldr + r_begin;
    float2* dst = xs + (size_t)d * ld;
#pragma unroll 4
    for (int cell = lane; cell < ncells; cell += 32) dst[cell] = __ldg(src + cell);
  }
}

// Raise a kernel's dynamic shared-memory limit (static plus dynamic shared
// memory above 48 KB needs it), once per device and size (set_bytes: per-device record of the limit already set,
// devices 0..63).  The check and the update run under one lock and only ever
// raise the limit, so that host threads launching the same kernel with
// different sizes cannot lower it under each other.
inline std::mutex& smem_attr_lock() {
  static std::mutex m;
  return m;
}

template <typename F>
cudaError_t ensure_smem(F* kern, size_t bytes, int* set_bytes /* [64] */) {
  // the default limit covers static plus dynamic shared memory up to 48 KB;
  // kernels here hold at most a few KB of static arrays
  if (bytes <= 32 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> guard(smem_attr_lock());
  if (set_bytes[dev] >= (int)bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set_bytes[dev] = (int)bytes;
  return e;
}

// CTAs of `kern` that fit on one SM with `threads` threads and `dyn_smem`
// bytes of dynamic shared memory: the smallest of the register, shared-memory
// and thread limits (from the kernel's attributes and the device's limits).
template <typename F>
int resident_ctas(F* kern, int threads, size_t dyn_smem) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 1;
  int dev = 0, regs_sm = 65536, smem_sm = 233472, thr_sm = 2048;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  }
  // registers are allocated per warp in units of 256
  const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = warp_regs > 0 ? regs_sm / (warp_regs * (threads / 32)) : 1;
  const size_t per_cta = dyn_smem + fa.sharedSizeBytes + 1024;   // 1 KB reserved per CTA
  const int by_smem = (int)(smem_sm / per_cta);
  const int by_thr = thr_sm / threads;
  int n = by_regs < by_smem ? by_regs : by_smem;
  n = n < by_thr ? n : by_thr;
  return n < 1 ? 1 : n;
}

}  // namespace stap
