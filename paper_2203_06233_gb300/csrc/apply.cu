// Weight application: output power of every range-Doppler cell,
//   out[s][k][r] = | w_{k, r/B, s}^H x_{k,r} |^2,
// the last step of the STAP kernel of arXiv 2203.06233 Sec. 4.2 (the adaptive
// filter output |w^H x|^2).
//
// Mapping: a CTA owns NBB consecutive training blocks of one Doppler bin (up
// to 256 range cells).  Their weights go to shared memory as [block][d][s]
// and their D x cells snapshot tile is staged by the same gather as the
// covariance kernel.  A thread owns one range cell and walks the steering
// vectors in chunks of SC, keeping SC complex accumulators in registers: per
// snapshot entry it reads x once and the chunk's weights as broadcast 16-byte
// loads, i.e. 1 + SC/2 shared loads for 4*SC FMAs.  Each output row
// out[s][k][cells] is written coalesced along range.
#include "batch.cuh"
#include "checked.cuh"
#include "snapshots.cuh"

namespace stap {
namespace {

constexpr int SC = 8;       // steering vectors per register chunk
constexpr int kThreads = 256;

// Parameters of one apply launch (one CPI); gx = the launch's grid.x.
struct ApplyParams {
  const float2* dop;
  const float2* wts;
  float* out;
  int C, K, R, ldr, T, B, S, NBB, CC;
  int gx;
};

__device__ __forceinline__ void apply_body(const ApplyParams& prm, int bx, int by) {
  const float2* __restrict__ dop = prm.dop;
  const float2* __restrict__ wts = prm.wts;
  float* __restrict__ out = prm.out;
  const int C = prm.C, K = prm.K, R = prm.R, ldr = prm.ldr, T = prm.T, B = prm.B, S = prm.S,
            NBB = prm.NBB, CC = prm.CC;
  extern __shared__ float4 sm4[];
  float2* sm = reinterpret_cast<float2*>(sm4);
  const int D = C * T;
  const int NB = R / B;
  const int k = by;
  const int b0 = bx * NBB;
  const int nbb = min(NBB, NB - b0);
  const int Sp = (S + SC - 1) / SC * SC;        // padded steering count (zero weights beyond S)
  float2* ws = sm;                              // [nbb][D][Sp]
  float2* xs = sm + (size_t)NBB * D * Sp;       // [D][CC + 1]
  const int ld = CC + 1;

  {  // weights of the nbb blocks, [j][d][s] in shared memory (zero for s >= S)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = warp; row < nbb * Sp; row += nw) {   // row = (block j, steering s)
      const int j = row / Sp, s = row - j * Sp;
      const float2* src = wts + (((size_t)k * NB + b0 + j) * S + s) * D;
      for (int d = lane; d < D; d += 32)
        ws[((size_t)j * D + d) * Sp + s] =
            (s < S && in_bounds((((long long)k * NB + b0 + j) * S + s) * D + d, (long long)K * NB * S * D,
                                kSiteApplyIn))
                ? __ldg(src + d) : make_float2(0.f, 0.f);
    }
  }
  const int cells = nbb * B;
  for (int c0 = 0; c0 < cells; c0 += CC) {
    const int cc = min(CC, cells - c0);
    __syncthreads();
    stage_snapshots(xs, ld, dop, C, K, ldr, T, k, b0 * B + c0, cc);
    __syncthreads();
    for (int rr = threadIdx.x; rr < cc; rr += blockDim.x) {
      const int j = (c0 + rr) / B;
      const float2* wj = ws + (size_t)j * D * Sp;
      const size_t r = (size_t)b0 * B + c0 + rr;
      for (int s0 = 0; s0 < S; s0 += SC) {
        float2 acc[SC];
#pragma unroll
        for (int q = 0; q < SC; ++q) acc[q] = make_float2(0.f, 0.f);
        for (int d = 0; d < D; ++d) {
          const float2 x = xs[d * ld + rr];
          const float4* w4 = reinterpret_cast<const float4*>(wj + (size_t)d * Sp + s0);
#pragma unroll
          for (int q = 0; q < SC / 2; ++q) {
            const float4 w = w4[q];      // weights s0+2q and s0+2q+1
            // acc += conj(w) * x
            acc[2 * q].x = fmaf(w.x, x.x, acc[2 * q].x);
            acc[2 * q].x = fmaf(w.y, x.y, acc[2 * q].x);
            acc[2 * q].y = fmaf(w.x, x.y, acc[2 * q].y);
            acc[2 * q].y = fmaf(-w.y, x.x, acc[2 * q].y);
            acc[2 * q + 1].x = fmaf(w.z, x.x, acc[2 * q + 1].x);
            acc[2 * q + 1].x = fmaf(w.w, x.y, acc[2 * q + 1].x);
            acc[2 * q + 1].y = fmaf(w.z, x.y, acc[2 * q + 1].y);
            acc[2 * q + 1].y = fmaf(-w.w, x.x, acc[2 * q + 1].y);
          }
        }
#pragma unroll
        for (int q = 0; q < SC; ++q)
          if (s0 + q < S && in_bounds(((long long)(s0 + q) * K + k) * ldr + (long long)r,
                                      ((long long)S * K - 1) * ldr + R, kSiteApplyOut))
            out[((size_t)(s0 + q) * K + k) * ldr + r] = fmaf(acc[q].x, acc[q].x, acc[q].y * acc[q].y);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads)
apply_kernel(ApplyParams p) {
  apply_body(p, blockIdx.x, blockIdx.y);
}

// the same apply as a persistent launch over the CPIs of a batch
__global__ void __launch_bounds__(kThreads)
apply_batched(BatchCtl ctl) {
  batched_loop<ApplyParams>(ctl, [&](const ApplyParams& p, int bx, int by, int) { apply_body(p, bx, by); });
}

// Register-resident form for small even D (the common shapes).  A thread owns
// two adjacent range cells: their 2 x D snapshot entries are loaded straight
// from the Doppler cube with one 16-byte load per entry (coalesced along
// range; T neighbouring bins are re-read through L2 by neighbouring CTAs) and
// stay in registers, while the weights of the CTA's blocks sit in shared
// memory as [block][s][d].  For each steering vector the thread reads its
// weights as D/2 broadcast 16-byte loads and does 8 D FMAs: FMA-bound.
// 128-thread CTAs: in a one-CPI run the apply of one range slab shares the
// SMs with the FP64 solves of others, and a smaller CTA takes fewer of a
// solve's warp slots (registers, shared memory) wherever it lands.
constexpr int kRegThreads = 128;
constexpr int kRegCells = 2 * kRegThreads;  // range cells per CTA

// registers: 64 while the snapshots fit, more for larger D
template <int D>
__device__ __forceinline__ void apply_reg_body(const ApplyParams& prm, int bx, int by) {
  const float2* __restrict__ dop = prm.dop;
  const float2* __restrict__ wts = prm.wts;
  float* __restrict__ out = prm.out;
  const int C = prm.C, K = prm.K, R = prm.R, ldr = prm.ldr, T = prm.T, B = prm.B, S = prm.S;
  extern __shared__ float4 sm4[];
  float2* ws = reinterpret_cast<float2*>(sm4);    // [nblk][S][D]
  const int NB = R / B;
  const int k = by;
  const int cta_r0 = bx * kRegCells;
  const int jb0 = cta_r0 / B;
  const int jb1 = min(NB - 1, (min(cta_r0 + kRegCells, R) - 1) / B);
  const int nblk = jb1 - jb0 + 1;
  {
    const float2* src = wts + ((size_t)k * NB + jb0) * S * D;
    const int n = nblk * S * D;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      ws[i] = in_bounds(((long long)k * NB + jb0) * S * D + i, (long long)K * NB * S * D, kSiteApplyIn)
                  ? __ldg(src + i) : make_float2(0.f, 0.f);
  }
  const int r0 = cta_r0 + 2 * threadIdx.x;
  float4 x[D];                                    // (cell r0, cell r0 + 1) per entry
  if (r0 < R) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int t = d / C, c = d - t * C;
      const int kk = wrap_bin(k + t - T / 2, K);
      const long long o = ((long long)c * K + kk) * ldr + r0;
      x[d] = in_bounds(o + 1, ((long long)C * K - 1) * ldr + R, kSiteApplyIn)
                 ? __ldg(reinterpret_cast<const float4*>(dop + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();
  if (r0 >= R) return;
  const int j = r0 / B - jb0;                      // B even: both cells in one block
  const float4* wj = reinterpret_cast<const float4*>(ws + (size_t)j * S * D);
  for (int s = 0; s < S; ++s) {
    float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll
    for (int d2 = 0; d2 < D / 2; ++d2) {
      const float4 w = wj[s * (D / 2) + d2];        // w_d = (w.x, w.y), w_{d+1} = (w.z, w.w)
      const float4 xa = x[2 * d2], xb = x[2 * d2 + 1];
      // acc += conj(w) * x for both cells
      a0r = fmaf(w.x, xa.x, a0r); a0r = fmaf(w.y, xa.y, a0r);
      a0i = fmaf(w.x, xa.y, a0i); a0i = fmaf(-w.y, xa.x, a0i);
      a1r = fmaf(w.x, xa.z, a1r); a1r = fmaf(w.y, xa.w, a1r);
      a1i = fmaf(w.x, xa.w, a1i); a1i = fmaf(-w.y, xa.z, a1i);
      a0r = fmaf(w.z, xb.x, a0r); a0r = fmaf(w.w, xb.y, a0r);
      a0i = fmaf(w.z, xb.y, a0i); a0i = fmaf(-w.w, xb.x, a0i);
      a1r = fmaf(w.z, xb.z, a1r); a1r = fmaf(w.w, xb.w, a1r);
      a1i = fmaf(w.z, xb.w, a1i); a1i = fmaf(-w.w, xb.z, a1i);
    }
    if (in_bounds(((long long)s * K + k) * ldr + r0 + 1, ((long long)S * K - 1) * ldr + R, kSiteApplyOut))
      *reinterpret_cast<float2*>(out + ((size_t)s * K + k) * ldr + r0) =
          make_float2(fmaf(a0r, a0r, a0i * a0i), fmaf(a1r, a1r, a1i * a1i));
  }
}

template <int D>
__global__ void __launch_bounds__(kRegThreads, D <= 12 ? 8 : (D <= 18 ? 6 : 4))
apply_reg_kernel(ApplyParams p) {
  apply_reg_body<D>(p, blockIdx.x, blockIdx.y);
}

template <int D>
__global__ void __launch_bounds__(kRegThreads, D <= 12 ? 8 : (D <= 18 ? 6 : 4))
apply_reg_batched(BatchCtl ctl) {
  batched_loop<ApplyParams>(ctl, [&](const ApplyParams& p, int bx, int by, int) {
    apply_reg_body<D>(p, bx, by);
  });
}

template <int D>
cudaError_t launch_apply_reg(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                             int ldr, int T, int B, int S, cudaStream_t s) {
  const int NB = R / B;
  const int max_blk = kRegCells / B + 2;
  const size_t smem = (size_t)(max_blk < NB ? max_blk : NB) * S * D * sizeof(float2);
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  cudaError_t e = ensure_smem(apply_reg_kernel<D>, smem, set_bytes);
  if (e == cudaSuccess) e = ensure_smem(apply_reg_batched<D>, smem, set_bytes_b);
  if (e != cudaSuccess) return e;
  dim3 grid((R + kRegCells - 1) / kRegCells, K);
  const ApplyParams p{dop, wts, out, C, K, R, ldr, T, B, S, 0, 0, (int)grid.x};
  return launch_params(reinterpret_cast<const void*>(apply_reg_kernel<D>),
                       reinterpret_cast<const void*>(apply_reg_batched<D>), grid, kRegThreads, smem, s, p);
}

}  // namespace

cudaError_t launch_apply(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                         int ldr, int T, int B, int S, cudaStream_t s, const Tune& tn) {
  const int D = C * T;
  const int NB = R / B;
  if (NB == 0) return cudaSuccess;
  // register-resident form: even D <= 24, even B and row stride (cell pairs
  // never straddle a block and 16-byte loads stay aligned), weights of a CTA
  // within 160 KB
  const bool aligned = (reinterpret_cast<uintptr_t>(dop) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(out) & 7) == 0 && ldr % 2 == 0;
  if (tn.apply_kind != 2 && aligned && D % 2 == 0 && D <= 24 && B % 2 == 0 &&
      (size_t)(kRegCells / B + 2) * S * D * sizeof(float2) <= 160 * 1024) {
    switch (D) {
      case 2: return launch_apply_reg<2>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 4: return launch_apply_reg<4>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 6: return launch_apply_reg<6>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 8: return launch_apply_reg<8>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 10: return launch_apply_reg<10>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 12: return launch_apply_reg<12>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 14: return launch_apply_reg<14>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 16: return launch_apply_reg<16>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 18: return launch_apply_reg<18>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 20: return launch_apply_reg<20>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 22: return launch_apply_reg<22>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      case 24: return launch_apply_reg<24>(dop, wts, out, C, K, R, ldr, T, B, S, s);
      default: break;
    }
  }
  constexpr size_t kBudget = 160 * 1024;
  const int Sp = (S + SC - 1) / SC * SC;
  int NBB = B >= kThreads ? 1 : kThreads / B;   // up to 256 cells per CTA
  if (NBB > NB) NBB = NB;
  auto wbytes = [&](int nbb) { return (size_t)nbb * D * Sp * sizeof(float2); };
  while (NBB > 1 && wbytes(NBB) > kBudget / 2) --NBB;
  if (wbytes(NBB) + (size_t)D * 2 * sizeof(float2) > kBudget) return cudaErrorInvalidValue;
  int CC = NBB * B;                              // cells staged per pass
  if (wbytes(NBB) + (size_t)D * (CC + 1) * sizeof(float2) > kBudget)
    CC = (int)((kBudget - wbytes(NBB)) / ((size_t)D * sizeof(float2))) - 1;
  const size_t smem = wbytes(NBB) + (size_t)D * (CC + 1) * sizeof(float2);
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  cudaError_t e = ensure_smem(apply_kernel, smem, set_bytes);
  if (e == cudaSuccess) e = ensure_smem(apply_batched, smem, set_bytes_b);
  if (e != cudaSuccess) return e;
  dim3 grid((NB + NBB - 1) / NBB, K);
  const ApplyParams p{dop, wts, out, C, K, R, ldr, T, B, S, NBB, CC, (int)grid.x};
  return launch_params(reinterpret_cast<const void*>(apply_kernel), reinterpret_cast<const void*>(apply_batched),
                       grid, kThreads, smem, s, p);
}

}  // namespace stap

namespace stap {
cudaError_t check_record_apply(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
