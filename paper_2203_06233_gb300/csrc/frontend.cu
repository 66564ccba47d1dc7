// Reduced-DOF front end (beyond the paper, whose cubes have 1000 channels):
// the N element channels of an element cube x[N][P][R] are combined into the
// C channels of the STAP cube by a matrix W[C][N],
//   y[c][p][r] = sum_{n<N} conj(W[c][n]) x[n][p][r],
// one chunk of Nc elements at a time (the first chunk writes y, later chunks
// add to it).
//
// HBM-bound: every element sample is read once per pass of CB = 4 output
// channels (one pass for C <= 4), y is read and written once per chunk.  A
// thread owns one (pulse, range) position, so a warp reads 32 consecutive
// complex samples of one element row (coalesced); W is read through L1 as a
// warp-wide broadcast.  Rounding: the elements of a chunk are summed in blocks
// of kBlk into a partial sum that is then added to the thread's total, which
// bounds the FP32 error growth by about (kBlk + Nc / kBlk) u instead of Nc u.
#include "stap_internal.cuh"

namespace stap {
namespace {

constexpr int kBlk = 32;
constexpr int kCB = 4;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
reduce_channels_kernel(const float2* __restrict__ x, const float2* __restrict__ W,
                       float2* __restrict__ y, int N, int n0, int Nc, int C, long long PR,
                       int accumulate) {
  const long long q = (long long)blockIdx.x * kThreads + threadIdx.x;   // (p, r)
  const int c0 = blockIdx.y * kCB;
  if (q >= PR) return;   // no barrier below
  float2 tot[kCB];
#pragma unroll
  for (int j = 0; j < kCB; ++j) tot[j] = make_float2(0.f, 0.f);
  for (int b0 = 0; b0 < Nc; b0 += kBlk) {
    const int b1 = min(Nc, b0 + kBlk);
    float2 part[kCB];
#pragma unroll
    for (int j = 0; j < kCB; ++j) part[j] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int n = b0; n < b1; ++n) {
      const float2 v = __ldg(x + (size_t)n * PR + q);
#pragma unroll
      for (int j = 0; j < kCB; ++j) {
        if (c0 + j < C) {   // uniform across the CTA
          const float2 w = __ldg(W + (size_t)(c0 + j) * N + n0 + n);
          // conj(w) v = (wr vr + wi vi) + i (wr vi - wi vr)
          part[j].x = fmaf(w.x, v.x, part[j].x);
          part[j].x = fmaf(w.y, v.y, part[j].x);
          part[j].y = fmaf(w.x, v.y, part[j].y);
          part[j].y = fmaf(-w.y, v.x, part[j].y);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kCB; ++j) {
      tot[j].x += part[j].x;
      tot[j].y += part[j].y;
    }
  }
#pragma unroll
  for (int j = 0; j < kCB; ++j) {
    if (c0 + j < C) {
      float2* dst = y + (size_t)(c0 + j) * PR + q;
      float2 o = tot[j];
      if (accumulate) {
        const float2 a = *dst;
        o.x = a.x + o.x;
        o.y = a.y + o.y;
      }
      *dst = o;
    }
  }
}

}  // namespace

cudaError_t launch_reduce_channels(const float2* x_chunk, const float2* W, float2* y, int N, int n0,
                                   int Nc, int C, int P, int R, bool accumulate, cudaStream_t s) {
  if (N < 1 || C < 1 || Nc < 1 || n0 < 0 || n0 + Nc > N) return cudaErrorInvalidValue;
  const long long PR = (long long)P * R;
  const long long blocks = (PR + kThreads - 1) / kThreads;
  const int cblocks = (C + kCB - 1) / kCB;
  if (blocks > 0x7fffffffLL || cblocks > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)blocks, (unsigned)cblocks);
  reduce_channels_kernel<<<grid, kThreads, 0, s>>>(x_chunk, W, y, N, n0, Nc, C, PR, accumulate ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace stap
