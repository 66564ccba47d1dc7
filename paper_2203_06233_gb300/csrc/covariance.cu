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
#include "df64.cuh"
#include "batch.cuh"
#include "checked.cuh"
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
covariance_ff_kernel(const float2* __restrict__ dop, double2* __restrict__ cov, int C, int K, int ldr,
                     int T, int B, int NB, int NS, int BC, double invB) {
  extern __shared__ float2 xs[];  // [NS][D][BC + 1]
  const int k = blockIdx.y;
  const int b0 = blockIdx.x * NS;
  const int D = C * T;
  const int E = D * (D + 1) / 2;
  const int ld = BC + 1;
  const int ns = min(NS, NB - b0);

  for (int c0 = 0; c0 < B; c0 += BC) {
    const int bc = min(BC, B - c0);
    __syncthreads();
    for (int j = 0; j < ns; ++j)
      stage_snapshots(xs + (size_t)j * D * ld, ld, dop, C, K, ldr, T, k, (b0 + j) * B + c0, bc);
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
      double vr = (ff::f2d_exact(re.s) + ff::f2d_exact(re.e)) * invB;
      double vi = (ff::f2d_exact(im.s) + ff::f2d_exact(im.e)) * invB;
      double2* out = cov + ((size_t)k * NB + b0 + j) * (size_t)D * D;
      if (c0 > 0) {  // later chunks add to what earlier chunks wrote (same thread owns the entry)
        const double2 prev = out[(size_t)i * D + l];
        vr += prev.x;
        vi += prev.y;
      }
      if (i == l) vi = 0.0;
      out[(size_t)i * D + l] = make_double2(vr, vi);
      if (i != l) out[(size_t)l * D + i] = make_double2(vr, ff::dneg(vi));
    }
  }
}

// ---------------------------------------------------------------------------
// Bin-pair form.  Block (t, t') of R_k is the cross-covariance of bins
// k + m_t and k + m_t' (m_t = t - floor(T/2)):
//   R_k[(t,c),(t',c')] = Q(k + m_t, k + m_t')[c][c'],
//   Q(k1, k2)[c][c'] = (1/B) sum_r X_c(k1, r) conj(X_c'(k2, r)),
// and Q(k2, k1) = Q(k1, k2)^H.  Neighbouring bins share these blocks, so a CTA
// that owns KT consecutive bins of one range block computes every Q(k1, k1+d),
// d < T, once (C(C+1)/2 entries for d = 0, C^2 otherwise) and assembles its KT
// covariances from them: T C^2 - C(C-1)/2 products per bin instead of
// D(D+1)/2.
//
// Accumulation on a fixed grid (error-free transformation in the manner of
// Rump, Ogita & Oishi, "Accurate floating-point summation part I", SISC 2008,
// ExtractScalar): for an entry whose row maxima are m1, m2 pick the power of
// two sig >= 4 B m1 m2.  For each product, s = fma(a, b, sig) rounds a*b onto
// the grid of sig, q = s - sig is exact, and the running sum of the q stays
// exact because every q lies on that grid and |sum| <= sig/2.  The remainder
// fma(a, b, -q) (|.| <= ulp(sig)/2) goes to a second FP32 accumulator.  Five
// FP32 instructions per real product; the pair is combined in FP64 at the end.
constexpr int kPairMaxThreads = 1024;   // one thread per Q entry, up to this

__device__ __forceinline__ float pow2_ceil(float x) {  // smallest power of two >= x
  if (!(x > 0.f)) return 1.0f;
  unsigned u = __float_as_uint(x);
  unsigned e = u >> 23;
  if (u & 0x7fffffu) e += 1;
  if (e < 1) e = 1;
  if (e > 254) e = 254;
  return __uint_as_float(e << 23);
}

__device__ __forceinline__ void grid_add(float& hi, float& lo, float a, float b, float sig) {
  const float s = __fmaf_rn(a, b, sig);
  const float q = __fsub_rn(s, sig);
  const float r = __fmaf_rn(a, b, -q);
  hi = __fadd_rn(hi, q);
  lo = __fadd_rn(lo, r);
}

// Parameters of one bin-pair launch (one CPI): grid gx = NB blocks by K / KT
// bin groups.
struct CovPairsParams {
  const float2* dop;
  double2* cov;
  int C, K, ldr, T, B, NB, KT, CB;
  double invB;
  int gx;
};

__device__ __forceinline__ void covariance_pairs_body(const CovPairsParams& prm, int bx, int by) {
  const float2* __restrict__ dop = prm.dop;
  double2* __restrict__ cov = prm.cov;
  const int C = prm.C, K = prm.K, ldr = prm.ldr, T = prm.T, B = prm.B, NB = prm.NB, KT = prm.KT,
            CB = prm.CB;
  const double invB = prm.invB;
  extern __shared__ double2 smd[];
  const int b = bx;
  const int k0 = by * KT;
  const int h = T / 2;
  const int NBIN = KT + T - 1;                    // staged bins k0-h .. k0+KT-1+(T-1-h)
  const int nrows = NBIN * C;
  const int ld = CB + 1;
  const int Ediag = C * (C + 1) / 2, Eoff = C * C;
  // items: d-major; d = 0 has NBIN * Ediag items, d > 0 has (NBIN - d) * Eoff
  const int nitems = NBIN * Ediag + (T - 1) * (2 * NBIN - T) / 2 * Eoff;
  double2* Q = smd;                                             // [nitems]
  float* m = reinterpret_cast<float*>(Q + nitems);              // [nrows] row maxima
  float2* X = reinterpret_cast<float2*>(m + ((nrows + 3) & ~3));  // [nrows][ld]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool pow2B = (B & (B - 1)) == 0;
  const float invBf = 1.0f / (float)B;

  // the B cells in chunks of CB: each chunk is summed error-free on its own
  // grid and added to Q in FP64
  for (int c0 = 0; c0 < B; c0 += CB) {
    const int cc = min(CB, B - c0);
    __syncthreads();
    for (int row = warp; row < nrows; row += nwarps) {   // rows (bin j, channel c)
      const int j = row / C, c = row - j * C;
      const int kk = wrap_bin(k0 - h + j, K);
      const float2* src = dop + ((size_t)c * K + kk) * ldr + (size_t)b * B + c0;
      float2* dst = X + row * ld;
      float mx = 0.f;
      for (int cell = lane; cell < cc; cell += 32) {
        const bool ok = in_bounds(((long long)c * K + kk) * ldr + (long long)b * B + c0 + cell,
                                  ((long long)C * K - 1) * ldr + (long long)NB * B, kSiteCovIn);
        const float2 x = ok ? __ldg(src + cell) : make_float2(0.f, 0.f);
        dst[cell] = x;
        mx = fmaxf(mx, fmaxf(fabsf(x.x), fabsf(x.y)));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) m[row] = mx;
    }
    __syncthreads();

    const float fourB = 4.0f * (float)cc;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
      int d = 0, rem = it;
      if (rem >= NBIN * Ediag) {
        rem -= NBIN * Ediag;
        d = 1;
        while (rem >= (NBIN - d) * Eoff) {
          rem -= (NBIN - d) * Eoff;
          ++d;
        }
      }
      int j1, c1, c2;
      if (d == 0) {
        j1 = rem / Ediag;
        unpack_lower(rem - j1 * Ediag, c1, c2);
      } else {
        j1 = rem / Eoff;
        const int e = rem - j1 * Eoff;
        c1 = e / C;
        c2 = e - c1 * C;
      }
      const int ra = j1 * C + c1, rb = (j1 + d) * C + c2;
      const float2* xa = X + ra * ld;
      const float2* xb = X + rb * ld;
      const float sig = pow2_ceil(fourB * m[ra] * m[rb]);
      float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;
#pragma unroll 4
      for (int cell = 0; cell < cc; ++cell) {
        const float2 a = xa[cell], bb = xb[cell];
        grid_add(hr, lr, a.x, bb.x, sig);
        grid_add(hr, lr, a.y, bb.y, sig);
        grid_add(hi, li, a.y, bb.x, sig);
        grid_add(hi, li, -a.x, bb.y, sig);
      }
      double2 v;
      if (pow2B) {  // 1/B is a power of two: scaling the pair in FP32 is exact
        v = make_double2(ff::f2d_exact(hr * invBf) + ff::f2d_exact(lr * invBf),
                         ff::f2d_exact(hi * invBf) + ff::f2d_exact(li * invBf));
      } else {
        v = make_double2((ff::f2d_exact(hr) + ff::f2d_exact(lr)) * invB, (ff::f2d_exact(hi) + ff::f2d_exact(li)) * invB);
      }
      if (c0 > 0) {
        const double2 p = Q[it];
        v.x += p.x;
        v.y += p.y;
      }
      Q[it] = v;
    }
  }
  __syncthreads();

  // assemble R_k for the KT bins of this tile
  const int D = C * T;
  auto qat = [&](int j1, int d, int c1, int c2) -> double2 {  // Q(bin j1, bin j1+d)[c1][c2]
    if (d == 0) {
      if (c1 >= c2) return Q[j1 * Ediag + c1 * (c1 + 1) / 2 + c2];
      const double2 v = Q[j1 * Ediag + c2 * (c2 + 1) / 2 + c1];
      return make_double2(v.x, ff::dneg(v.y));
    }
    // blocks d' < d come first: NBIN Ediag + sum_{e=1}^{d-1} (NBIN - e) Eoff
    const int off = NBIN * Ediag + Eoff * ((d - 1) * NBIN - d * (d - 1) / 2);
    return Q[off + j1 * Eoff + c1 * C + c2];
  };
  for (int idx = threadIdx.x; idx < KT * D * D; idx += blockDim.x) {
    const int kl = idx / (D * D);
    const int e = idx - kl * D * D;
    const int i = e / D, l = e - i * D;
    const int t1 = i / C, c1 = i - t1 * C, t2 = l / C, c2 = l - t2 * C;
    double2 v;
    if (t1 <= t2) {
      v = qat(kl + t1, t2 - t1, c1, c2);
    } else {
      const double2 w = qat(kl + t2, t1 - t2, c2, c1);
      v = make_double2(w.x, ff::dneg(w.y));
    }
    if (i == l) v.y = 0.0;
    const long long o = (((long long)(k0 + kl) * NB + b) * D + i) * D + l;
    if (in_bounds(o, (long long)K * NB * D * D, kSiteCovOut)) cov[o] = v;
  }
}

__global__ void __launch_bounds__(kPairMaxThreads)
covariance_pairs_kernel(CovPairsParams p) {
  covariance_pairs_body(p, blockIdx.x, blockIdx.y);
}

// the same covariances as a persistent launch over the CPIs of a batch
__global__ void __launch_bounds__(kPairMaxThreads)
covariance_pairs_batched(BatchCtl ctl) {
  batched_loop<CovPairsParams>(ctl, [&](const CovPairsParams& p, int bx, int by, int) {
    covariance_pairs_body(p, bx, by);
  });
}

}  // namespace

cudaError_t launch_covariance_fp32(const float2* dop, double2* cov, int C, int K, int R, int ldr,
                                   int T, int B, cudaStream_t s, const Tune& tn) {
  const int D = C * T;
  const int E = D * (D + 1) / 2;
  const int NB = R / B;
  if (NB == 0) return cudaSuccess;
  // bin-pair kernel: the B cells of KT + T - 1 bins in shared memory, in
  // chunks of CB cells when the whole block does not fit
  {
    constexpr size_t kPairBudget = 200 * 1024;
    auto pair_smem = [&](int kt, int cb) {
      const int nbin = kt + T - 1;
      const size_t nitems = (size_t)nbin * (C * (C + 1) / 2) +
                            (size_t)(T - 1) * (2 * nbin - T) / 2 * C * C;
      const size_t nrows = (size_t)nbin * C;
      return nitems * sizeof(double2) + ((nrows + 3) & ~(size_t)3) * sizeof(float) +
             nrows * (cb + 1) * sizeof(float2);
    };
    int KT = K < 16 ? K : 16;  // K is a power of two, so KT divides it
    while (KT > 1 && pair_smem(KT, B) > kPairBudget) KT >>= 1;
    if (tn.cov_kt > 0 && tn.cov_kt <= K && K % tn.cov_kt == 0 && pair_smem(tn.cov_kt, B) <= kPairBudget)
      KT = tn.cov_kt;
    int CB = B;
    while (CB > 32 && pair_smem(KT, CB) > kPairBudget) CB = (CB + 1) / 2;
    if (pair_smem(KT, CB) <= kPairBudget) {
      const size_t smem = pair_smem(KT, CB);
      static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
      cudaError_t e = ensure_smem(covariance_pairs_kernel, smem, set_bytes);
      if (e == cudaSuccess) e = ensure_smem(covariance_pairs_batched, smem, set_bytes_b);
      if (e != cudaSuccess) return e;
      dim3 grid(NB, K / KT);
      // Many Q entries (large C): one thread per entry, rounded up to whole
      // warps (at most 32 warps, rounds balanced above that), so that they
      // are not spread unevenly over a last, partly idle round of threads.
      // Few entries: 256 threads, which share the SMs better with the solve
      // kernels of other range slabs.
      const int nbin = KT + T - 1;
      const int nitems = nbin * (C * (C + 1) / 2) + (T - 1) * (2 * nbin - T) / 2 * C * C;
      int threads = 256;
      if (nitems > 512) {
        const int rounds = (nitems + kPairMaxThreads - 1) / kPairMaxThreads;
        threads = ((nitems + rounds - 1) / rounds + 31) / 32 * 32;
        if (threads > kPairMaxThreads) threads = kPairMaxThreads;
      }
      const CovPairsParams p{dop, cov, C, K, ldr, T, B, NB, KT, CB, 1.0 / (double)B, (int)grid.x};
      return launch_params(reinterpret_cast<const void*>(covariance_pairs_kernel),
                           reinterpret_cast<const void*>(covariance_pairs_batched), grid, threads, smem,
                           s, p);
    }
  }
  // general form: one tile per system, cells in chunks
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
  return launch_or_defer(s, [=](cudaStream_t st) {
    covariance_ff_kernel<<<grid, 256, smem, st>>>(dop, cov, C, K, ldr, T, B, NB, NS, BC, 1.0 / (double)B);
    return cudaGetLastError();
  });
}

}  // namespace stap

namespace stap {
cudaError_t check_record_covariance(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
