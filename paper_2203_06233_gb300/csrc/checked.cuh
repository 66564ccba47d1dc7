// Bounds checks of the checked build (libstap compiled with -DSTAP_CHECKED).
//
// Every kernel index into a global buffer (and, in the tensor-core kernels,
// into shared and tensor memory) is compared with the extent of that buffer
// as the launch sees it: in_bounds(i, n, site) is true for 0 <= i < n.
// Otherwise the violation is counted, the first one in each source file is
// recorded (site code, index, extent) in a device record of that file, and
// the caller skips the access.  Nothing traps: a checked run always finishes
// and stap_check_report reads the records.  In the normal build in_bounds is
// the constant true and every check compiles away.
#pragma once

#include "stap_internal.cuh"

namespace stap {

// What a checked access was (stap_check_report's site code).
enum CheckSite : int {
  kSiteDopplerIn = 1,    // cube samples read by the Doppler transform
  kSiteDopplerOut = 2,   // Doppler output written
  kSiteCovIn = 3,        // Doppler samples read by the covariance
  kSiteCovOut = 4,       // covariance entries written
  kSiteSolveIn = 5,      // covariance entries read by a solve kernel
  kSiteSolveOut = 6,     // weights written
  kSiteApplyIn = 7,      // Doppler samples or weights read by the apply
  kSiteApplyOut = 8,     // output power written
  kSiteTcIn = 9,         // global operand read by a tensor-core kernel
  kSiteTcOut = 10,       // global result written by a tensor-core kernel
  kSiteTcSmem = 11,      // shared-memory operand offset of a tensor-core kernel
  kSiteTcTmem = 12,      // tensor-memory column read by a tensor-core epilogue
  kSiteTrain = 13,       // training-matrix entry read or written
};

namespace {

#ifdef STAP_CHECKED
__device__ CheckRecord g_check;   // one per source file (internal linkage)

__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_check.count, 1ULL) == 0ULL) {
    g_check.index = i;
    g_check.extent = n;
    g_check.site = site;
  }
  return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, int) { return true; }
#endif

// Copy this file's record to *out and clear it (zeros in the normal build).
inline cudaError_t read_check_record(CheckRecord* out) {
#ifdef STAP_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(out, g_check, sizeof(CheckRecord));
  if (e != cudaSuccess) return e;
  const CheckRecord zero{};
  return cudaMemcpyToSymbol(g_check, &zero, sizeof(CheckRecord));
#else
  *out = CheckRecord{};
  return cudaSuccess;
#endif
}

}  // namespace
}  // namespace stap
