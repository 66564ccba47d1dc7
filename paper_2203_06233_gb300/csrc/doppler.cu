// Doppler transform (statement T of the STAP kernel, arXiv 2203.06233 Sec. 4.2):
//   dop[c][k][r] = sum_{p<P} h[p] cube[c][p][r] exp(-2 pi i p k / K),  K >= P,
// computed as a zero-padded length-K FFT over the pulse axis.
//
// Layout: the pulse axis has stride ldr (the full range extent; a launch may
// cover R <= ldr cells of it), the range axis is contiguous.  A CTA
// owns one channel and TR (8-32) consecutive range cells and does TR independent
// length-K FFTs by the four-step split K = N1 * N2:
//   input  index n = n1 + N1 n2,   output index k = k2 + N2 k1,
//   Y[n1][k2] = W_K^{n1 k2} * sum_{n2} x[n1 + N1 n2] W_{N2}^{n2 k2}     (pass A)
//   X[k2 + N2 k1] = sum_{n1} Y[n1][k2] W_{N1}^{n1 k1}                    (pass B)
// Each thread does one short FFT in registers per pass; the only shared-memory
// traffic is the Y transpose between the passes.  Global loads (pass A) and
// stores (pass B) are coalesced along range: a warp touches runs of TR
// consecutive complex samples of pulse/bin rows.  The window and the zero
// padding are applied while loading.  HBM traffic is the algorithmic minimum:
// 8*C*P*R bytes read + 8*C*K*R bytes written.
//
// PRI-staggered snapshots: TW sub-windows of PW = P - TW + 1 pulses per
// channel, sub-window t covering the pulses t .. t+PW-1 with the window
// h'[n - t] (length PW) and the pulses' own phase exp(-j 2 pi n k / K), i.e. the
// same zero-padded FFT of the window-shifted pulse train; sub-window t of
// channel c is written as output row t*C + c.  CTA row y = c*TW + t, so the TW
// transforms of one channel run back to back and re-read its pulses from L2.
// (TW = 1, PW = P: the plain transform.)
#include "batch.cuh"
#include "checked.cuh"
#include "snapshots.cuh"

namespace stap {
namespace {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

__host__ __device__ constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// In-register radix-2 FFT of length N (forward, natural order in and out).
// tw[m] = W_K^m; W_N^j = tw[j * (K / N)].
template <int N, int K>
__device__ __forceinline__ void fft_reg(float2 (&v)[N], const float2* __restrict__ tw) {
  constexpr int LOGN = ilog2c(N);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev(i, LOGN);
    if (i < j) {
      float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float2 w = tw[j * (K / len)];
#pragma unroll
      for (int st = 0; st < N; st += len) {
        const float2 a = v[st + j];
        const float2 b = (j == 0) ? v[st + j + half] : cmulf(v[st + j + half], w);
        v[st + j] = make_float2(a.x + b.x, a.y + b.y);
        v[st + j + half] = make_float2(a.x - b.x, a.y - b.y);
      }
    }
  }
}

// Parameters of one launch (one CPI): grid gx = ceil(R / TR) range tiles by
// C * TW rows.
struct DopplerParams {
  const float2* cube;
  float2* dop;
  const float* win;
  const float2* tw;
  int P, R, ldr, C, TW, PW;
  int gx;
};

template <int LOGK, int TR>
__device__ __forceinline__ void doppler_body(const DopplerParams& prm, int bx, int by) {
  const float2* __restrict__ cube = prm.cube;
  float2* __restrict__ dop = prm.dop;
  const float* __restrict__ win = prm.win;
  const float2* __restrict__ twg = prm.tw;
  const int P = prm.P, R = prm.R, ldr = prm.ldr, C = prm.C, TW = prm.TW, PW = prm.PW;
  constexpr int K = 1 << LOGK;
  constexpr int N1 = 1 << ((LOGK + 1) / 2);
  constexpr int N2 = 1 << (LOGK / 2);
  extern __shared__ float2 smem[];
  float2* tw = smem;        // [K]
  float2* Y = smem + K;     // [N1][N2][TR]

  const int tid = threadIdx.x;
  const int c = by / TW, t = by - c * TW;   // channel, sub-window
  const int r0 = bx * TR;
  for (int m = tid; m < K; m += blockDim.x) tw[m] = twg[m];

  // ---- pass A: thread (col, n1), N2-point FFT over n2 ----
  {
    const int col = tid % TR, n1 = tid / TR;
    const int r = r0 + col;
    const bool in_range = r < R;
    const float2* src = cube + (size_t)c * P * ldr + r;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int n = n1 + N1 * n2;
      float2 x = make_float2(0.f, 0.f);
      if (in_range && n >= t && n < t + PW &&
          in_bounds((long long)c * P * ldr + r + (long long)n * ldr, (long long)(C * P - 1) * ldr + R,
                    kSiteDopplerIn)) {
        x = __ldg(src + (size_t)n * ldr);
        const float h = __ldg(win + (n - t));
        x.x *= h;
        x.y *= h;
      }
      v[n2] = x;
    }
    __syncthreads();  // twiddle table ready
    fft_reg<N2, K>(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const float2 y = (k2 == 0) ? v[k2] : cmulf(v[k2], tw[n1 * k2]);
      Y[(n1 * N2 + k2) * TR + col] = y;
    }
  }
  __syncthreads();

  // ---- pass B: thread (col, k2), N1-point FFT over n1 ----
  if (tid < TR * N2) {
    const int col = tid % TR, k2 = tid / TR;
    const int r = r0 + col;
    float2 u[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = Y[(n1 * N2 + k2) * TR + col];
    fft_reg<N1, K>(u, tw);
    if (r < R) {
      float2* dst = dop + ((size_t)t * C + c) * K * ldr + r;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1)
        if (in_bounds(((long long)t * C + c) * K * ldr + r + (long long)(k2 + N2 * k1) * ldr,
                      ((long long)C * TW * K - 1) * ldr + R, kSiteDopplerOut))
          dst[(size_t)(k2 + N2 * k1) * ldr] = u[k1];
    }
  }
}

template <int LOGK, int TR>
__global__ void __launch_bounds__(TR * (1 << ((LOGK + 1) / 2)))
doppler_fft_kernel(DopplerParams p) {
  doppler_body<LOGK, TR>(p, blockIdx.x, blockIdx.y);
}

// the same transform as a persistent launch over the CPIs of a batch
template <int LOGK, int TR>
__global__ void __launch_bounds__(TR * (1 << ((LOGK + 1) / 2)))
doppler_fft_batched(BatchCtl ctl) {
  batched_loop<DopplerParams>(ctl, [&](const DopplerParams& p, int bx, int by, int) {
    doppler_body<LOGK, TR>(p, bx, by);
  });
}

template <int LOGK, int TR>
cudaError_t launch_logk_tr(const float2* cube, float2* dop, const float* win, const float2* tw, int C,
                           int TW, int P, int R, int ldr, cudaStream_t s) {
  constexpr int K = 1 << LOGK;
  constexpr int N1 = 1 << ((LOGK + 1) / 2);
  const size_t smem = (size_t)K * sizeof(float2) * (1 + TR);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  cudaError_t e = ensure_smem(doppler_fft_kernel<LOGK, TR>, smem, set_bytes);
  if (e == cudaSuccess) e = ensure_smem(doppler_fft_batched<LOGK, TR>, smem, set_bytes_b);
  if (e != cudaSuccess) return e;
  dim3 grid((R + TR - 1) / TR, C * TW);
  const DopplerParams p{cube, dop, win, tw, P, R, ldr, C, TW, P - TW + 1, (int)grid.x};
  return launch_params(reinterpret_cast<const void*>(doppler_fft_kernel<LOGK, TR>),
                       reinterpret_cast<const void*>(doppler_fft_batched<LOGK, TR>), grid, TR * N1,
                       smem, s, p);
}

// range cells per CTA: by default 256-thread CTAs (TR * N1) of at most 32
// columns, so that several CTAs fit per SM; a warp still covers >= 64
// contiguous bytes of a row (two full 32-byte sectors)
template <int LOGK>
cudaError_t launch_logk(const float2* cube, float2* dop, const float* win, const float2* tw, int C,
                        int TW, int P, int R, int ldr, cudaStream_t s, int tr) {
  constexpr int N1 = 1 << ((LOGK + 1) / 2);
  if (tr == 0) tr = (N1 >= 32) ? 8 : (N1 >= 16 ? 16 : 32);
  switch (tr) {
    case 8: return launch_logk_tr<LOGK, 8>(cube, dop, win, tw, C, TW, P, R, ldr, s);
    case 16: return launch_logk_tr<LOGK, 16>(cube, dop, win, tw, C, TW, P, R, ldr, s);
    case 32: return launch_logk_tr<LOGK, 32>(cube, dop, win, tw, C, TW, P, R, ldr, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_doppler(const float2* cube, float2* dop, const float* win, const float2* tw,
                           int C, int TW, int P, int K, int R, int ldr, cudaStream_t s, const Tune& t) {
  const int tr = t.dop_tr;
  if (TW < 1 || TW > P || (long long)C * TW > 65535) return cudaErrorInvalidValue;
  switch (ilog2c(K)) {
    case 0: return launch_logk<0>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 1: return launch_logk<1>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 2: return launch_logk<2>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 3: return launch_logk<3>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 4: return launch_logk<4>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 5: return launch_logk<5>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 6: return launch_logk<6>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 7: return launch_logk<7>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 8: return launch_logk<8>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 9: return launch_logk<9>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    case 10: return launch_logk<10>(cube, dop, win, tw, C, TW, P, R, ldr, s, tr);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stap

namespace stap {
cudaError_t check_record_doppler(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
