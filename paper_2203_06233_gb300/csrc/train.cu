// Training with guard cells (an option beyond the paper's own-block training,
// which leaves the cell under test in its training data): the covariance that
// block b's weights use is the mean of the covariances of the adjacent blocks
// b-1 and b+1, or the one of them that exists at either end of the range, so
// that the cell under test and the other cells of its own block act as guard
// cells.  With equal block sizes the mean of two sample covariances is the
// sample covariance of their 2B cells.
//
// Memory-bound: reads two c128 matrices and writes one per system (in 16-byte
// elements, coalesced along the flattened [K][NB][D][D] index); the halving is
// exact.
//
// The sliding window below generalises it: a guard band of `guard` groups on
// each side of the group under test and `half` training groups beyond it on
// each side (guard 0, half 1 is the neighbour-block form).
#include "batch.cuh"
#include "checked.cuh"
#include "stap_internal.cuh"

namespace stap {
namespace {

__global__ void __launch_bounds__(256)
train_neighbours_kernel(const double2* __restrict__ in, double2* __restrict__ out, int NB,
                        long long DD, long long total) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long sys = idx / DD;
    const int b = (int)(sys % NB);
    const bool lo = b > 0, hi = b + 1 < NB;
    double2 v;
    if (lo && hi && in_bounds(idx - DD, total, kSiteTrain) && in_bounds(idx + DD, total, kSiteTrain)) {
      const double2 p = __ldg(in + idx - DD), q = __ldg(in + idx + DD);
      v = make_double2((p.x + q.x) * 0.5, (p.y + q.y) * 0.5);
    } else {
      const long long src = idx + (lo ? -DD : DD);
      v = in_bounds(src, total, kSiteTrain) ? __ldg(in + src) : make_double2(0.0, 0.0);
    }
    out[idx] = v;
  }
}

// Sliding training window: group j (B cells) takes the mean of the
// covariances of the groups j-guard-half .. j-guard-1 and j+guard+1 ..
// j+guard+half that exist, summed left side first in increasing group order
// and then divided component by component by their count -- the same
// operations in the same order as the definition, so the result is exact to
// the last bit.  One thread per (k, j, entry), entries fastest (coalesced);
// neighbouring groups read overlapping windows, which the L2 serves.
__global__ void __launch_bounds__(256)
train_window_kernel(const double2* __restrict__ in, double2* __restrict__ out, int NB,
                    long long DD, long long total, int guard, int half) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long sys = idx / DD;
    const int j = (int)(sys % NB);
    const long long e = idx - sys * DD;
    const double2* base = in + (sys - j) * DD + e;   // group 0 of this bin, entry e
    double re = 0.0, im = 0.0;
    int count = 0;
    for (int side = 0; side < 2; ++side) {
      const int i0 = side == 0 ? j - guard - half : j + guard + 1;
      for (int m = 0; m < half; ++m) {
        const int i = i0 + m;
        if (i < 0 || i >= NB) continue;
        const double2 v = in_bounds((sys - j + i) * DD + e, total, kSiteTrain) ? __ldg(base + (long long)i * DD)
                                                                               : make_double2(0.0, 0.0);
        re += v.x;
        im += v.y;
        ++count;
      }
    }
    out[idx] = make_double2(re / (double)count, im / (double)count);
  }
}

}  // namespace

cudaError_t launch_train_window(const double2* in, double2* out, int K, int NB, int D, int guard,
                                int half, cudaStream_t s) {
  if (guard < 0 || half < 1 || NB < 2 * guard + 2) return cudaErrorInvalidValue;
  const long long DD = (long long)D * D;
  const long long total = (long long)K * NB * DD;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  return launch_or_defer(s, [=](cudaStream_t st) {
    train_window_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, out, NB, DD, total, guard, half);
    return cudaGetLastError();
  });
}

cudaError_t launch_train_neighbours(const double2* in, double2* out, int K, int NB, int D,
                                    cudaStream_t s) {
  if (NB < 2) return cudaErrorInvalidValue;
  const long long DD = (long long)D * D;
  const long long total = (long long)K * NB * DD;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  return launch_or_defer(s, [=](cudaStream_t st) {
    train_neighbours_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, out, NB, DD, total);
    return cudaGetLastError();
  });
}

}  // namespace stap

namespace stap {
cudaError_t check_record_train(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
