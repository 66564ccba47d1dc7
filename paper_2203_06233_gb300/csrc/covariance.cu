// Covariance per (Doppler bin, range training block) (statement U of the STAP
// kernel, arXiv 2203.06233 Sec. 4.2, read as the sample covariance):
//   cov[k][b] = (1/B) sum_{r in block b} x_{k,r} x_{k,r}^H
// with x_{k,r} the D = C*T snapshot of T adjacent Doppler bins.
//
// Precision: the solve downstream sees covariances whose condition number is
// bounded only by the diagonal load (about 1e3 * D), so rounding R to FP32
// would dominate the weight error.  Each entry is therefore accumulated
// error-free in FP32 pairs: every product a*b is split exactly into p + e by
// one FMA (TwoProduct), p is added to the running sum with Knuth's TwoSum, and
// all rounding errors are collected in a second FP32 accumulator.  The result
// sum + errors is accurate to about n^2 u^2 times the sum of |terms|
// (Ogita, Rump & Oishi, "Accurate sum and dot product", SISC 2005, Dot2),
// far below FP32 rounding, and is written as FP64.  All of this runs on the
// FP32 pipe (about 10 FP32 ops per real product); only the final conversion
// touches FP64.
//
// Mapping: a CTA owns NS consecutive blocks of one Doppler bin, stages their
// D x B snapshot tiles in shared memory (chunks of BC cells if B is large) and
// gives each thread whole entries (i >= l) of the lower triangle; the upper
// triangle is written as the conjugate mirror.
#include "snapshots.cuh"

namespace stap {
namespace {

struct FF {
  float s, e;  // value = s + e (e collects every rounding error)
};

__device__ __forceinline__ void ff_add_prod(FF& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);        // a*b = p + pe exactly
  const float t = __fadd_rn(acc.s, p);         // TwoSum(acc.s, p) = t + te exactly
  const float z = __fsub_rn(t, acc.s);
  const float te = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, z)), __fsub_rn(p, z));
  acc.s = t;
  acc.e = __fadd_rn(acc.e, __fadd_rn(te, pe));
}

__device__ __forceinline__ void unpack_lower(int q, int& i, int& l) {
  int r = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > q) --r;
  while ((r + 1) * (r + 2) / 2 <= q) ++r;
  i = r;
  l = q - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(256)
covariance_ff_kernel(const float2* __restrict__ dop, double2* __restrict__ cov, int C, int K, int R,
                     int T, int B, int NB, int NS, int BC) {
  extern __shared__ float2 xs[];  // [NS][D][BC + 1]
  const int k = blockIdx.y;
  const int b0 = blockIdx.x * NS;
  const int D = C * T;
  const int E = D * (D + 1) / 2;
  const int ld = BC + 1;
  const int ns = min(NS, NB - b0);
  const double invB = 1.0 / (double)B;

  for (int c0 = 0; c0 < B; c0 += BC) {
    const int bc = min(BC, B - c0);
    __syncthreads();
    for (int j = 0; j < ns; ++j)
      stage_snapshots(xs + (size_t)j * D * ld, ld, dop, C, K, R, T, k, (b0 + j) * B + c0, bc);
    __syncthreads();
    for (int it = threadIdx.x; it < ns * E; it += blockDim.x) {
      const int j = it / E;
      int i, l;
      unpack_lower(it - j * E, i, l);
      const float2* xi = xs + ((size_t)j * D + i) * ld;
      const float2* xl = xs + ((size_t)j * D + l) * ld;
      FF re{0.f, 0.f}, im{0.f, 0.f};
      for (int rr = 0; rr < bc; ++rr) {
        const float2 a = xi[rr], b = xl[rr];
        // a * conj(b) = (a.x b.x + a.y b.y) + i (a.y b.x - a.x b.y)
        ff_add_prod(re, a.x, b.x);
        ff_add_prod(re, a.y, b.y);
        ff_add_prod(im, a.y, b.x);
        ff_add_prod(im, -a.x, b.y);
      }
      double vr = ((double)re.s + (double)re.e) * invB;
      double vi = ((double)im.s + (double)im.e) * invB;
      double2* out = cov + ((size_t)k * NB + b0 + j) * (size_t)D * D;
      if (c0 > 0) {  // later chunks add to what earlier chunks wrote (same thread owns the entry)
        const double2 prev = out[(size_t)i * D + l];
        vr += prev.x;
        vi += prev.y;
      }
      if (i == l) vi = 0.0;
      out[(size_t)i * D + l] = make_double2(vr, vi);
      if (i != l) out[(size_t)l * D + i] = make_double2(vr, -vi);
    }
  }
}

}  // namespace

cudaError_t launch_covariance_fp32(const float2* dop, double2* cov, int C, int K, int R, int T,
                                   int B, cudaStream_t s) {
  const int D = C * T;
  const int E = D * (D + 1) / 2;
  const int NB = R / B;
  constexpr size_t kSmemBudget = 96 * 1024;
  int BC = B;
  if ((size_t)D * (BC + 1) * sizeof(float2) > kSmemBudget)
    BC = (int)(kSmemBudget / ((size_t)D * sizeof(float2))) - 1;
  if (BC < 1) return cudaErrorInvalidValue;
  int NS = E >= 256 ? 1 : 256 / E;
  NS = min(NS, NB);
  while (NS > 1 && (size_t)NS * D * (BC + 1) * sizeof(float2) > kSmemBudget) --NS;
  const size_t smem = (size_t)NS * D * (BC + 1) * sizeof(float2);
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(covariance_ff_kernel, smem, set_bytes);
  if (e != cudaSuccess) return e;
  dim3 grid((NB + NS - 1) / NS, K);
  covariance_ff_kernel<<<grid, 256, smem, s>>>(dop, cov, C, K, R, T, B, NB, NS, BC);
  return cudaGetLastError();
}

}  // namespace stap
