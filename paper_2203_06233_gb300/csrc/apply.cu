// Weight application: output power of every range-Doppler cell,
//   out[s][k][r] = | w_{k, r/B, s}^H x_{k,r} |^2,
// the last step of the STAP kernel of arXiv 2203.06233 Sec. 4.2 (the adaptive
// filter output |w^H x|^2).
//
// Mapping: a CTA owns one (Doppler bin k, block b) system.  Its S x D weights
// go to shared memory transposed ([d][s]) and its D x B snapshot tile is
// staged by the same gather as the covariance kernel.  A thread owns one range
// cell and SB consecutive steering vectors: per snapshot entry it reads x once
// and SB weights as broadcasts, so shared-memory traffic is one read per FMA
// pair.  Output rows are written coalesced along range.
#include "snapshots.cuh"

namespace stap {
namespace {

constexpr int SB = 4;  // steering vectors per thread

__global__ void __launch_bounds__(256)
apply_kernel(const float2* __restrict__ dop, const float2* __restrict__ wts, float* __restrict__ out,
             int C, int K, int R, int T, int B, int S, int BC) {
  extern __shared__ float2 sm[];
  const int D = C * T;
  const int NB = R / B;
  const int b = blockIdx.x, k = blockIdx.y;
  const int ld = BC + 1;
  float2* ws = sm;                     // [D][S]
  float2* xs = sm + (size_t)D * S;     // [D][ld]
  const float2* wsrc = wts + ((size_t)k * NB + b) * S * D;
  for (int idx = threadIdx.x; idx < S * D; idx += blockDim.x) {
    const int s = idx / D, d = idx - s * D;
    ws[d * S + s] = __ldg(wsrc + idx);
  }
  const int ngroups = (S + SB - 1) / SB;
  for (int c0 = 0; c0 < B; c0 += BC) {
    const int bc = min(BC, B - c0);
    __syncthreads();
    stage_snapshots(xs, ld, dop, C, K, R, T, k, b * B + c0, bc);
    __syncthreads();
    for (int it = threadIdx.x; it < bc * ngroups; it += blockDim.x) {
      const int g = it / bc, rr = it - g * bc;
      const int s0 = g * SB;
      float2 acc[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q) acc[q] = make_float2(0.f, 0.f);
      for (int d = 0; d < D; ++d) {
        const float2 x = xs[d * ld + rr];
        const float2* wd = ws + d * S + s0;
#pragma unroll
        for (int q = 0; q < SB; ++q) {
          if (s0 + q < S) {
            const float2 w = wd[q];
            // acc += conj(w) * x
            acc[q].x = fmaf(w.x, x.x, acc[q].x);
            acc[q].x = fmaf(w.y, x.y, acc[q].x);
            acc[q].y = fmaf(w.x, x.y, acc[q].y);
            acc[q].y = fmaf(-w.y, x.x, acc[q].y);
          }
        }
      }
      const size_t r = (size_t)b * B + c0 + rr;
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        if (s0 + q < S)
          out[((size_t)(s0 + q) * K + k) * R + r] = fmaf(acc[q].x, acc[q].x, acc[q].y * acc[q].y);
      }
    }
  }
}

}  // namespace

cudaError_t launch_apply(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                         int T, int B, int S, cudaStream_t s) {
  const int D = C * T;
  const int NB = R / B;
  if (NB == 0) return cudaSuccess;
  constexpr size_t kBudget = 96 * 1024;
  const size_t wbytes = (size_t)D * S * sizeof(float2);
  if (wbytes + (size_t)D * 2 * sizeof(float2) > kBudget) return cudaErrorInvalidValue;
  int BC = B;
  if (wbytes + (size_t)D * (BC + 1) * sizeof(float2) > kBudget)
    BC = (int)((kBudget - wbytes) / ((size_t)D * sizeof(float2))) - 1;
  const size_t smem = wbytes + (size_t)D * (BC + 1) * sizeof(float2);
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(apply_kernel, smem, set_bytes);
  if (e != cudaSuccess) return e;
  dim3 grid(NB, K);
  apply_kernel<<<grid, 256, smem, s>>>(dop, wts, out, C, K, R, T, B, S, BC);
  return cudaGetLastError();
}

}  // namespace stap
