// Persistent batched launches (the batch of uneven CPIs, a8).
//
// A kernel whose body takes its block coordinates as arguments runs either
// as an ordinary launch (one CPI, coordinates from blockIdx) or as a
// persistent launch over many CPIs at once: each CTA repeatedly takes the
// next virtual block g from an atomic counter, finds the CPI whose range of
// virtual blocks holds g (prefix sums over the CPIs, binary search), loads
// that CPI's parameter block and runs the body on the block's coordinates.
// The CTAs never wait on one another: a CTA stops when the counter passes
// the last virtual block.  The host side records, instead of issuing, each
// CPI's launch (the launchers pick kernel, shape and parameters as for a
// single CPI), groups the records of one kernel class and issues one
// persistent launch per group.
#pragma once

#include <cstring>
#include <functional>
#include <vector>

#include "stap_internal.cuh"

namespace stap {

// Parameters of one persistent launch, in device memory: `params` holds n
// parameter blocks of `stride` bytes (a multiple of 16, the array 16-byte
// aligned); prefix[i] is the first virtual block of CPI i (prefix[n] = the
// total); *counter starts at 0.
struct BatchCtl {
  const unsigned char* params;
  const long long* prefix;
  unsigned long long* counter;
  int n;
  int stride;
};

// The per-CTA scheduling loop.  body(params, bx, by, gx) runs one virtual
// block of a CPI whose grid is gx x gy (gx taken from the parameter block).
template <class P, class Body>
__device__ __forceinline__ void batched_loop(const BatchCtl& ctl, Body&& body) {
  __shared__ long long s_g;
  const long long total = ctl.prefix[ctl.n];
  for (;;) {
    __syncthreads();                    // the previous item is done with s_g
    if (threadIdx.x == 0) s_g = (long long)atomicAdd(ctl.counter, 1ULL);
    __syncthreads();
    const long long g = s_g;
    if (g >= total) break;
    int lo = 0, hi = ctl.n;             // prefix[lo] <= g < prefix[lo + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(ctl.prefix + mid) <= g) lo = mid;
      else hi = mid;
    }
    const P p = *reinterpret_cast<const P*>(ctl.params + (size_t)lo * ctl.stride);
    const long long local = g - __ldg(ctl.prefix + lo);
    body(p, (int)(local % p.gx), (int)(local / p.gx), p.gx);
  }
}

// ---- host side ----------------------------------------------------------------

constexpr int kMaxParamBytes = 256;

// One recorded launch of one CPI.
struct LaunchRecord {
  const void* single = nullptr;     // the ordinary kernel, taking (P)
  const void* batched = nullptr;    // its persistent twin, taking (BatchCtl), or nullptr
  dim3 grid;                        // the ordinary grid
  long long vblocks = 0;            // virtual blocks of the persistent twin (gx x gy of its body)
  int block = 0;
  size_t smem = 0;
  int psize = 0;
  alignas(16) unsigned char params[kMaxParamBytes];
  // a launch without a persistent twin: issued as recorded, on the given stream
  std::function<cudaError_t(cudaStream_t)> replay;
};

// While a recorder is installed on this host thread, the launchers below
// append their launches to it instead of issuing them.
struct LaunchRecorder {
  std::vector<LaunchRecord> records;
};
LaunchRecorder*& current_recorder();

// Issue (or record) an ordinary launch of `single` with one parameter block.
// vblocks: the body's virtual blocks (default grid.x * grid.y; a grid-stride
// kernel passes its work units, with p.gx set to match).
template <class P>
cudaError_t launch_params(const void* single, const void* batched, dim3 grid, int block, size_t smem,
                          cudaStream_t s, const P& p, long long vblocks = -1) {
  static_assert(sizeof(P) <= kMaxParamBytes, "parameter block too large");
  if (LaunchRecorder* rec = current_recorder()) {
    LaunchRecord r;
    r.single = single;
    r.batched = batched;
    r.grid = grid;
    r.block = block;
    r.smem = smem;
    r.vblocks = vblocks >= 0 ? vblocks : (long long)grid.x * grid.y;
    r.psize = (int)sizeof(P);
    std::memcpy(r.params, &p, sizeof(P));
    rec->records.push_back(r);
    return cudaSuccess;
  }
  void* args[] = {const_cast<P*>(&p)};
  return cudaLaunchKernel(single, grid, dim3(block), args, smem, s);
}

// Issue (or record, to be issued later in the same order) a launch that has
// no persistent twin.
template <class F>
cudaError_t launch_or_defer(cudaStream_t s, F&& issue) {
  if (LaunchRecorder* rec = current_recorder()) {
    LaunchRecord r;
    r.replay = std::function<cudaError_t(cudaStream_t)>(issue);
    rec->records.push_back(std::move(r));
    return cudaSuccess;
  }
  return issue(s);
}

}  // namespace stap
