// Mixed-precision contractions on the tensor cores (tcgen05): the covariance
// (statement U of the paper's STAP kernel, Sec. 4.2) and the weight
// application, as split products with FP32 accumulation in TMEM.  Three
// arithmetics (stap_precision):
//   TF32X3  kind::tf32.  x = hi + lo, hi = tf32(x), lo = tf32(x - hi);
//           products hi*hi + hi*lo + lo*hi (about 2^-21 relative each).
//   BF16X3  kind::f16 on bf16.  x = hi + mid + lo, each piece the bf16
//           rounding of what the earlier pieces leave (x - hi and
//           x - hi - mid are exact in FP32); the six products whose piece
//           orders sum to at most 2 (hi*hi, hi*mid, mid*hi, hi*lo, mid*mid,
//           lo*hi), about 2^-24 relative each.
//   FP16S   kind::f16 on fp16 with per-block scaling.  Every value of a
//           block (one covariance system; one apply tile of 128 cells, and
//           each weight vector) is multiplied by one power of two 2^e that
//           brings the block's largest magnitude into [2^14, 2^15), well
//           inside fp16's range; then x 2^e = hi + lo (fp16 pieces, about 22
//           significant bits down to 2^-18 of the block maximum) and the
//           products are hi*hi + hi*lo + lo*hi.  The epilogue removes the
//           scales exactly (powers of two).
//
// Covariance.  R = (1/B) X X^H per (Doppler bin, range block) with X the
// D x B snapshot tile, X = Xr + j Xi.  The operand rows are stacked as
// Y = [Xr ; Xi] for G systems at once (D8 = D rounded up
// to 8; rows of entries a >= D are zero): rows 0 .. G D8 - 1 hold Xr of the
// G systems, rows G D8 .. 2 G D8 - 1 their Xi.  Accumulators of NA = G D8
// rounded up to 16 columns, M = 128, in one of two forms:
//   stacked (D8 <= 64, G = floor(64 / D8)): A is all 128 rows [Xr ; Xi], and
//     two MMAs per product and K step give every block of the tile:
//       Xr-rows x Xr -> [XrXr^T ; XiXr^T],   Xr-rows x Xi -> [XrXi^T ; XiXi^T]
//     in 2 NA <= 128 TMEM columns (two CTAs per SM).  TMEM lane GD + i holds
//     the Xi row of the entry whose Xr row is lane i; the epilogue hands the
//     Xi rows to the Xr lanes through shared memory;
//   split (D8 > 64, G = 1): four MMAs per product and K step into four
//     accumulators XrXr, XiXi, XiXr, XrXi (512 columns, one CTA per SM).
//   Re R = XrXr + XiXi and Im R = XiXr - XrXi are formed in the epilogue.
//   Each accumulator holds one product, so it takes one MMA step per K step
//   and product: the tensor cores' FP32 accumulation loses up to about an
//   ulp of the running sum per step, and summing Re R in one accumulator
//   (twice the steps) measurably doubled the covariance error.
// TMEM lane i (entry a of system g) holds its row of each block in columns
// g D8 + l.  Only the blocks between different systems (G > 1) are
// computed and not used.  Each snapshot element is loaded once, split once
// and stored once per piece (the B operand is the A operand's own rows).
// Thread a writes R[a][l] for l >= a as conj into row l, column a, so a
// warp's stores of one output row are contiguous; the full Hermitian form
// (the ABI call) mirrors the same value into row a, so it is Hermitian bit
// for bit.
//
// Apply.  out[s][k][r] = |w_{k,b(r),s}^H x_{k,r}|^2 per tile of 128 range
// cells of one bin: M = 128 cells, K = 2 D (the snapshot's re/im pairs in
// memory order), N = two rows per (block j, steering s) of the tile:
//   [wr_0, wi_0, wr_1, wi_1, ...] -> Re y,  [-wi_0, wr_0, -wi_1, wr_1, ...] -> Im y.
// One accumulator; lane m (cell r0 + m) reads the columns of its own block.
//
// Pipeline per CTA (256 threads, persistent over tiles): the operand chunk
// is staged into one of two shared-memory stages (K-major core matrices, no
// swizzle) by all threads, thread 0 issues the chunk's MMAs and commits them
// to that stage's mbarrier, and the next chunk is staged into the other
// stage meanwhile.  Waits are bounded: a pipeline wait gives up after
// wait_polls polls; the CTA then records a timeout, waits (bounded by
// kDefaultWaitPolls) for the MMAs it still has in flight, frees its TMEM and
// stops.  A stage whose wait gave up stays pending, so that drain covers it.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "df64.cuh"
#include "batch.cuh"
#include "checked.cuh"
#include "snapshots.cuh"
#include "tcgen05.cuh"

namespace stap {
namespace {

enum { kTF32X3 = 0, kBF16X3 = 1, kFP16S = 2 };

template <int PREC>
struct Fmt;
template <>
struct Fmt<kTF32X3> {
  static constexpr int NPC = 2, ESZ = 4, KI = 8, NPROD = 3;
};
template <>
struct Fmt<kBF16X3> {
  static constexpr int NPC = 3, ESZ = 2, KI = 16, NPROD = 6;
};
template <>
struct Fmt<kFP16S> {
  static constexpr int NPC = 2, ESZ = 2, KI = 16, NPROD = 3;
};

// pieces (A, B) of the products kept, leading product first
__device__ __forceinline__ int prod_a(int i) { return i < 3 ? (i == 2 ? 1 : 0) : (i == 3 ? 0 : (i == 4 ? 1 : 2)); }
__device__ __forceinline__ int prod_b(int i) { return i < 3 ? (i == 1 ? 1 : 0) : (i == 3 ? 2 : (i == 4 ? 1 : 0)); }

constexpr int kThreads = 256;                 // 8 warps stage; warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kWaitIter = kDefaultWaitPolls;  // drain waits before TMEM is freed

// ---- splitting ---------------------------------------------------------------

// TF32 pieces of one value
__device__ __forceinline__ void split_tf32(float x, uint32_t (&w)[2]) {
  w[0] = tc::to_tf32(x);
  w[1] = tc::to_tf32(x - __uint_as_float(w[0]));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
__device__ __forceinline__ uint32_t pack_f16(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// bf16 pieces hi, mid, lo of a pair (a in the low half of each word)
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t (&w)[3]) {
  const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
  const float ar = a - __bfloat162float(ah), br = b - __bfloat162float(bh);   // exact
  const __nv_bfloat16 am = __float2bfloat16_rn(ar), bm = __float2bfloat16_rn(br);
  const float ar2 = ar - __bfloat162float(am), br2 = br - __bfloat162float(bm);   // exact
  w[0] = pack_bf16(ah, bh);
  w[1] = pack_bf16(am, bm);
  w[2] = pack_bf16(__float2bfloat16_rn(ar2), __float2bfloat16_rn(br2));
}

// fp16 pieces hi, lo of a pair already scaled into fp16's range
__device__ __forceinline__ void split_f16(float a, float b, uint32_t (&w)[2]) {
  const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
  w[0] = pack_f16(ah, bh);
  w[1] = pack_f16(__float2half_rn(a - __half2float(ah)), __float2half_rn(b - __half2float(bh)));
}

// Power of two 2^e with m 2^e in [2^14, 2^15) for a block maximum m (1 for a
// zero or non-finite maximum; non-finite inputs then propagate).
__device__ __forceinline__ float block_scale(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  int E = 0;
  frexpf(m, &E);              // m = f 2^E, f in [1/2, 1)
  int e = 15 - E;
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return ldexpf(1.f, e);
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int PREC>
__device__ __forceinline__ void issue_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  if constexpr (PREC == kTF32X3)
    tc::mma_tf32(d, a, b, idesc, acc);
  else
    tc::mma_f16(d, a, b, idesc, acc);
}

template <int PREC>
__host__ __device__ constexpr uint32_t idesc_for(int N) {
  return PREC == kTF32X3 ? tc::idesc_tf32(128, N) : tc::idesc_f16(128, N, PREC == kBF16X3);
}

// ---- covariance -----------------------------------------------------------------

// Two forms (see the file header): stacked (STK, D8 <= 64: M spans [Xr ; Xi]
// of G = floor(64 / D8) systems, two accumulators of NA <= 64 columns) and
// split (D8 > 64: four accumulators, 512 columns).  A piece of a stage holds
// ROWS operand rows of RB bytes (16 KB either way).
constexpr int kCovU = 8;                      // staging units per warp and chunk (<= 64 units / 8 warps)
constexpr int kCovPiece = 16384;              // bytes of one piece of one stage

template <bool STK>
struct CovForm {
  static constexpr int RB = STK ? 128 : 64;   // bytes of one operand row per chunk
  static constexpr int ROWS = kCovPiece / RB; // 128 (stacked) or 256 (split) rows
  static constexpr int NCM = RB / 16;         // core matrices along K per chunk
  static constexpr int COLS = STK ? 128 : 512;   // TMEM columns of a tile
  static constexpr int GROWS = STK ? 64 : 128;   // rows of Xr a tile takes (G D8 <= GROWS)
};

template <int PREC>
constexpr size_t cov_smem() { return 2 * (size_t)Fmt<PREC>::NPC * kCovPiece; }

template <int PREC, bool STK>
__global__ void __launch_bounds__(kThreads, 2)
covariance_tcx_kernel(const float2* __restrict__ dop, double2* __restrict__ cov, int C, int K,
                      int ldr, int T, int B, int NB, int D8, int G, long long ntiles, int lower_only,
                      DeviceStatus* __restrict__ status, int wait_polls) {
  using F = Fmt<PREC>;
  using Fm = CovForm<STK>;
  constexpr int KC = Fm::RB / F::ESZ;        // cells per chunk
  constexpr int SBO = 8 * Fm::RB;            // bytes between 8-row groups
  constexpr int STAGE = F::NPC * kCovPiece;
  constexpr int CPW = 16 / F::ESZ;           // cells per core-matrix row
  constexpr int CPL = CPW / 4;               // cells per lane in a staging unit
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ long long rowbase[128];          // dop offset of Xr/Xi row p, or -1
  __shared__ float sscale[128];               // per system scale (FP16S)
  __shared__ int smax[128];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = C * T;
  const int GD = G * D8;                     // Xr rows of the tile (Xi rows follow)
  const int NA = (GD + 15) / 16 * 16;        // columns of one accumulator
  const long long nsys = (long long)K * NB;
  const int nchunks = (B + KC - 1) / KC;
  const int units = (GD / 8) * Fm::NCM;      // row groups x core matrices along K

  for (int i = tid; i < 2 * STAGE / 4; i += kThreads) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (warp == 0) tc::tmem_alloc(&tmem_base, Fm::COLS);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_for<PREC>(NA);
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  long long gch = 0;                          // chunks issued by this CTA (stage = gch & 1)

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long sys0 = tile * G;
    if (tid < GD) {  // row p = g D8 + a: entry a of system sys0 + g
      long long base = -1;
      const int g = tid / D8, a = tid - g * D8;
      const long long sys = sys0 + g;
      if (a < D && sys < nsys) {
        const int k = (int)(sys / NB), b = (int)(sys - (long long)k * NB);
        const int t = a / C, c = a - t * C;
        base = ((long long)c * K + wrap_bin(k + t - T / 2, K)) * ldr + (long long)b * B;
      }
      rowbase[tid] = base;
    }
    if (PREC == kFP16S && tid < G) smax[tid] = 0;
    __syncthreads();
    if constexpr (PREC == kFP16S) {   // each system's largest |re|, |im| over its B cells
      // two rows per warp and pass, so that both rows' loads are in flight together
      for (int p0 = warp; p0 < GD; p0 += 2 * (kThreads / 32)) {
        const int p1 = p0 + kThreads / 32;
        const long long base0 = rowbase[p0], base1 = p1 < GD ? rowbase[p1] : -1;
        float m0 = 0.f, m1 = 0.f;
#pragma unroll 4
        for (int j = lane; j < B; j += 32) {
          if (base0 >= 0) {
            const float2 x = __ldg(dop + base0 + j);
            m0 = fmaxf(m0, fmaxf(fabsf(x.x), fabsf(x.y)));
          }
          if (base1 >= 0) {
            const float2 x = __ldg(dop + base1 + j);
            m1 = fmaxf(m1, fmaxf(fabsf(x.x), fabsf(x.y)));
          }
        }
        m0 = warp_max(m0);
        m1 = warp_max(m1);
        if (lane == 0) {   // m >= 0: int order
          atomicMax(&smax[p0 / D8], __float_as_int(m0));
          if (p1 < GD) atomicMax(&smax[p1 / D8], __float_as_int(m1));
        }
      }
      __syncthreads();
      if (tid < G) sscale[tid] = block_scale(__int_as_float(smax[tid]));
      __syncthreads();
    }
    // A unit is one core matrix (8 rows x 16 bytes) of the Xr rows and the
    // matching one of the Xi rows; lane l takes row 8 rg + l/4 and CPL cells
    // and writes one 32-bit word per piece into each.  Warp w takes units
    // w, w + 8, ... (at most kCovU of them).  The next chunk's loads are
    // issued before this chunk's barrier and MMAs, so their latency overlaps
    // both.
    // Per tile, each lane's unit uu covers row (warp + 8 uu) / NCM * 8 + l/4
    // (its dop offset and, for FP16S, its system's scale fetched here once)
    // and the same cells of every chunk ((warp % NCM) CPW + (l & 3) CPL on).
    long long rbase[kCovU];
    float rsc[kCovU];
#pragma unroll
    for (int uu = 0; uu < kCovU; ++uu) {
      const int unit = warp + uu * (kThreads / 32);
      const int p = (unit / Fm::NCM) * 8 + (lane >> 2);
      rbase[uu] = unit < units ? rowbase[p] : -1;
      rsc[uu] = (PREC == kFP16S && unit < units) ? sscale[p / D8] : 1.f;
    }
    const int jl = (warp % Fm::NCM) * CPW + (lane & 3) * CPL;
    float2 v[kCovU][CPL];
    auto load_chunk = [&](int ch) {
      const int c0 = ch * KC;
#pragma unroll
      for (int uu = 0; uu < kCovU; ++uu) {
        const int j = c0 + jl;
        const long long base = rbase[uu];
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc)
          v[uu][cc] = (base >= 0 && j + cc < B &&
                       in_bounds(base + j + cc, ((long long)C * K - 1) * ldr + (long long)NB * B, kSiteTcIn))
                          ? __ldg(dop + base + j + cc) : make_float2(0.f, 0.f);
      }
    };
    if (ok) load_chunk(0);
    for (int ch = 0; ch < nchunks && ok; ++ch, ++gch) {
      const int st = (int)(gch & 1);
      uint8_t* stage = sm + st * STAGE;
      if (pending[st]) {  // the MMAs that last read this stage must be done
        ok = tc::mbar_wait(&mbar[st], parity[st], wait_polls);
        if (ok) {
          parity[st] ^= 1u;
          pending[st] = false;
        }
      }
      ok = __syncthreads_and(ok);
      if (!ok) break;
#pragma unroll
      for (int uu = 0; uu < kCovU; ++uu) {
        const int unit = warp + uu * (kThreads / 32);
        if (unit >= units) continue;
        const int rg = unit / Fm::NCM, cmk = unit % Fm::NCM;
        const int off = rg * SBO + cmk * 128 + (lane >> 2) * 16 + (lane & 3) * 4;
        const int offi = off + (GD / 8) * SBO;
        if (!in_bounds(offi + 3, kCovPiece, kSiteTcSmem)) continue;   // the word's last byte
        if constexpr (PREC == kTF32X3) {
          uint32_t wr[2], wi[2];
          split_tf32(v[uu][0].x, wr);
          split_tf32(v[uu][0].y, wi);
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) {
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + off) = wr[pc];
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + offi) = wi[pc];
          }
        } else if constexpr (PREC == kBF16X3) {
          uint32_t wr[3], wi[3];
          split_bf16(v[uu][0].x, v[uu][1].x, wr);
          split_bf16(v[uu][0].y, v[uu][1].y, wi);
#pragma unroll
          for (int pc = 0; pc < 3; ++pc) {
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + off) = wr[pc];
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + offi) = wi[pc];
          }
        } else {
          const float sc = rsc[uu];
          uint32_t wr[2], wi[2];
          split_f16(v[uu][0].x * sc, v[uu][1].x * sc, wr);
          split_f16(v[uu][0].y * sc, v[uu][1].y * sc, wi);
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) {
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + off) = wr[pc];
            *reinterpret_cast<uint32_t*>(stage + pc * kCovPiece + offi) = wi[pc];
          }
        }
      }
      if (ch + 1 < nchunks) load_chunk(ch + 1);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t base = tc::smem_u32(stage);
        const uint32_t bot = (uint32_t)(GD / 8) * SBO;   // the Xi rows
#pragma unroll
        for (int ks = 0; ks < KC / F::KI; ++ks) {
          const uint32_t o = ks * 256;
#pragma unroll
          for (int pr = 0; pr < F::NPROD; ++pr) {
            const uint32_t pa = base + prod_a(pr) * kCovPiece + o;
            const uint32_t pb = base + prod_b(pr) * kCovPiece + o;
            const bool acc = !(ch == 0 && ks == 0 && pr == 0);
            const uint64_t ar = tc::smem_desc(pa, 128, SBO);
            const uint64_t br = tc::smem_desc(pb, 128, SBO), bi = tc::smem_desc(pb + bot, 128, SBO);
            if constexpr (STK) {   // A = [Xr ; Xi] (all 128 rows)
              issue_mma<PREC>(tmem, ar, br, idesc, acc);                // [XrXr^T ; XiXr^T]
              issue_mma<PREC>(tmem + NA, ar, bi, idesc, acc);           // [XrXi^T ; XiXi^T]
            } else {
              const uint64_t ai = tc::smem_desc(pa + bot, 128, SBO);
              issue_mma<PREC>(tmem, ar, br, idesc, acc);                // Xr Xr^T
              issue_mma<PREC>(tmem + NA, ai, bi, idesc, acc);           // Xi Xi^T
              issue_mma<PREC>(tmem + 2 * NA, ai, br, idesc, acc);       // Xi Xr^T
              issue_mma<PREC>(tmem + 3 * NA, ar, bi, idesc, acc);       // Xr Xi^T
            }
          }
        }
        tc::mma_commit(&mbar[st]);
      }
      pending[st] = true;
    }
    // all MMAs of this tile done (commits complete in order; drain both stages)
    for (int s2 = 0; s2 < 2; ++s2) {
      if (pending[s2] && ok) {
        ok = tc::mbar_wait(&mbar[s2], parity[s2], wait_polls);
        if (ok) {
          parity[s2] ^= 1u;
          pending[s2] = false;
        }
      }
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows i of the
    // tile); warps w and w + 4 take alternate column blocks of 8
    const int q4 = warp & 3, hf = warp >> 2;
    const uint32_t lb = (uint32_t)(q4 * 32) << 16;
    const float invB = 1.f / (float)B;
    const int LDX = D8 + 1;                    // exchange row pitch (floats; odd: no bank conflicts)
    float* xir = reinterpret_cast<float*>(sm);  // stacked: XiXr rows (the stages are idle now)
    float* xii = xir + GD * LDX;                //          XiXi rows
    if constexpr (STK) {
      // lanes GD .. 2 GD - 1 hold the Xi rows: [XiXr | XiXi] of entry a of
      // system g in columns g D8 + l; hand them to the Xr lanes through
      // shared memory
      if (q4 * 32 < 2 * GD && q4 * 32 + 32 > GD) {   // warp-uniform
        const int ii = q4 * 32 + lane - GD;
        const bool xi = ii >= 0 && ii < GD;
        const int g = xi ? ii / D8 : 0, a = ii - g * D8;
        for (int cb = hf * 8; cb < NA; cb += 16) {
          float x0[8], x1[8];
          in_bounds(NA + cb + 7, Fm::COLS, kSiteTcTmem);   // recorded only
          tc::tmem_ld8x2(tmem + lb + cb, tmem + lb + NA + cb, x0, x1);
          if (xi && a < D) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int l = cb + u - g * D8;
              if (l >= 0 && l < D && in_bounds(ii * LDX + l, GD * LDX, kSiteTcSmem)) {
                xir[ii * LDX + l] = x0[u];
                xii[ii * LDX + l] = x1[u];
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if (q4 * 32 < GD) {   // warps holding Xr rows (warp-uniform)
      const int i = q4 * 32 + lane;
      const int g = i / D8, a = i - g * D8;
      const long long sys = sys0 + g;
      const bool mine = i < GD && a < D && sys < nsys;
      const float sc = (PREC == kFP16S && i < GD) ? 1.f / sscale[g] : 1.f;   // exact
      double2* out = cov + (size_t)(mine ? sys : 0) * D * D;
      const int gw0 = (q4 * 32) / D8;
      const int gw1 = min(G - 1, (q4 * 32 + 31) / D8);
      for (int gg = gw0; gg <= gw1; ++gg) {
        for (int cb = hf * 8; cb < D8; cb += 16) {   // warp-uniform bounds
          // one system per tile: a block of columns left of the warp's first
          // row has no l >= a entry
          if (G == 1 && cb + 8 <= q4 * 32) continue;
          float re8[8], im8[8];
          const uint32_t tcol = tmem + lb + gg * D8 + cb;
          if constexpr (STK) {
            float xrxi[8];
            in_bounds(NA + gg * D8 + cb + 7, Fm::COLS, kSiteTcTmem);   // recorded only
            tc::tmem_ld8x2(tcol, tcol + NA, re8, xrxi);
            if (mine && g == gg) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int l = cb + u;
                const int xo = i * LDX + l;   // this lane's own row (entries l < a or l >= D unused)
                re8[u] += xii[xo];             // XrXr + XiXi
                im8[u] = xir[xo] - xrxi[u];    // XiXr - XrXi
              }
            }
          } else {
            in_bounds(3 * NA + gg * D8 + cb + 7, Fm::COLS, kSiteTcTmem);   // recorded only
            float ii8[8], ri8[8];
            tc::tmem_ld8x2(tcol, tcol + NA, re8, ii8);
            tc::tmem_ld8x2(tcol + 2 * NA, tcol + 3 * NA, im8, ri8);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              re8[u] += ii8[u];
              im8[u] -= ri8[u];
            }
          }
          if (mine && g == gg) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int l = cb + u;
              if (l >= a && l < D) {   // R[a][l], stored conjugated at [l][a]
                const float re = re8[u] * sc * sc * invB;
                const float im = l == a ? 0.f : im8[u] * sc * sc * invB;
                const double dre = ff::f2d_exact(re), dim = ff::f2d_exact(im);
                const long long ext = nsys * D * D, o = sys * D * D;
                if (in_bounds(o + (long long)l * D + a, ext, kSiteTcOut))
                  out[(size_t)l * D + a] = make_double2(dre, ff::dneg(dim));   // sign bit: no FP64 op
                if (!lower_only && l != a && in_bounds(o + (long long)a * D + l, ext, kSiteTcOut))
                  out[(size_t)a * D + l] = make_double2(dre, dim);
              }
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM and exchange reads done before the next tile overwrites them
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicExch(&status->timeout, 1u);
    for (int s2 = 0; s2 < 2; ++s2)      // let MMAs still in flight finish (bounded)
      if (pending[s2]) tc::mbar_wait(&mbar[s2], parity[s2], kWaitIter);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, Fm::COLS);
}

// ---- apply ------------------------------------------------------------------------

constexpr int kAppRB = 64;                    // bytes of one operand row per chunk (4 core matrices)
constexpr int kAppA = 128 * kAppRB;           // A piece: 128 cells (8 KB)
constexpr int kAppB = 256 * kAppRB;           // B piece: at most 256 weight rows (16 KB)
constexpr int kAppU = 16;                     // staging units per warp and chunk: (64 A + at most 64 B units) / 8 warps

// two stages of the pieces of 128 cell rows and NP weight rows
template <int PREC>
constexpr size_t apply_smem(int NP) { return 2 * (size_t)Fmt<PREC>::NPC * (kAppA + (size_t)NP * kAppRB); }

template <int PREC>
__global__ void __launch_bounds__(kThreads, 2)   // two CTAs per SM (TMEM <= 256 columns each)
apply_tcx_kernel(const float2* __restrict__ dop, const float2* __restrict__ wts,
                 float* __restrict__ out, int C, int K, int R, int ldr, int T, int B, int S, int NB,
                 int NP, int tmem_cols, long long ntiles, DeviceStatus* __restrict__ status,
                 int wait_polls) {
  using F = Fmt<PREC>;
  constexpr int KC = kAppRB / F::ESZ;         // K elements per chunk: 16 (tf32) or 32 (16-bit)
  constexpr int SBO = 8 * kAppRB;
  constexpr int NCM = kAppRB / 16;            // core matrices along K per chunk
  const int PIECE = kAppA + NP * kAppRB;      // cell rows, then NP weight rows
  const int STAGE = F::NPC * PIECE;
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ long long colbase[128];          // dop offset of snapshot entry d's row
  __shared__ long long wbase[256];            // wts offset of weight row n (vector n/2), or -1
  __shared__ float wsc[128];                  // per weight vector scale (FP16S)
  __shared__ float winv[128];                 // its inverse times the tile's (exact: powers of two)
  __shared__ float xsc_s;
  __shared__ int xmax;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = C * T;
  const int K2 = 2 * D;
  const int tiles_per_k = (R + 127) / 128;
  const int nbt = B < 128 ? 128 / B : 1;
  const int Nq = nbt * S;                     // weight vectors per tile
  const int nchunks = (K2 + KC - 1) / KC;
  // A units: one core matrix of 8 cell rows; B units: a pair of core
  // matrices along K of one 8-row group (4 weight vectors), each lane one
  // weight element written to the vector's two rows
  const int unitsA = 16 * NCM, units = unitsA + (NP / 8) * (NCM / 2);

  for (int i = tid; i < 2 * STAGE / 4; i += kThreads) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (warp == 0) tc::tmem_alloc(&tmem_base, tmem_cols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_for<PREC>(NP);
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  long long gch = 0;

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int k = (int)(tile / tiles_per_k);
    const int r0 = (int)(tile - (long long)k * tiles_per_k) * 128;
    const int b0 = r0 / B;
    if (tid < D) {
      const int t = tid / C, c = tid - t * C;
      colbase[tid] = ((long long)c * K + wrap_bin(k + t - T / 2, K)) * ldr;
    }
    {
      const int q = tid >> 1, j = q / S, s = q - j * S;
      wbase[tid] = (tid < NP && q < Nq && b0 + j < NB) ? ((((long long)k * NB + b0 + j) * S + s) * D) : -1;
    }
    if (PREC == kFP16S && tid == 0) xmax = 0;
    __syncthreads();
    if constexpr (PREC == kFP16S) {   // the tile's largest |x| component, each vector's largest |w|
      float m = 0.f;
      const int rn = min(128, R - r0);
#pragma unroll 8
      for (int e = tid; e < D * 128; e += kThreads) {   // entry d = e / 128 of cell e % 128
        const int d = e >> 7, mm = e & 127;
        if (mm < rn) {
          const float2 v = __ldg(dop + colbase[d] + r0 + mm);
          m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
      }
      m = warp_max(m);
      if (lane == 0) atomicMax(&xmax, __float_as_int(m));
      for (int q = warp; q < Nq; q += kThreads / 32) {
        const long long wb = wbase[2 * q];
        float mw = 0.f;
        if (wb >= 0)
          for (int d = lane; d < D; d += 32) {
            const float2 w = __ldg(wts + wb + d);
            mw = fmaxf(mw, fmaxf(fabsf(w.x), fabsf(w.y)));
          }
        mw = warp_max(mw);
        if (lane == 0) wsc[q] = block_scale(mw);
      }
      __syncthreads();
      const float xs = block_scale(__int_as_float(xmax));
      if (tid == 0) xsc_s = xs;
      if (tid < Nq) winv[tid] = 1.f / (wsc[tid] * xs);   // powers of two: exact
      __syncthreads();
    }
    // K elements kap0 .. kap0 + KC - 1 of the A rows (cells) and of the B
    // rows (weights).  An A unit is one core matrix: lane l takes row
    // 8 rg + l/4 and K elements 4 cm + (l & 3) (tf32) or one re/im pair
    // (16-bit).  A B unit is two core matrices cm = 2 j + h (h = l / 16) of
    // one 8-row group: lane l takes weight vector 4 rg + (l / 4) % 4 and word
    // l & 3 of both its rows, [wr, wi] (even) and [-wi, wr] (odd), from one
    // load and one split (pieces of -x are minus those of x).  Warp w takes
    // units w, w + 8, ... (at most kAppU); the next chunk's loads are issued
    // before this chunk's barrier and MMAs.
    // With NCM = 4 the 64 A units are units 0-63: warp w's unit uu < 8 is
    // row group (w >> 2) + 2 uu, core matrix w & 3.  Its B unit vb (unit
    // 64 + w + 8 vb) is row group (w >> 1) + 4 vb, core matrices 2 (w & 1) + h.
    // Row offsets, weight-vector offsets and scales are fixed per tile; the
    // snapshot entry and the weight element per chunk.
    static_assert(NCM == 4 && kAppU == 16, "unit layout");
    constexpr int kAU = 8, kBU = kAppU - kAU;
    const int unitsB = units - unitsA;
    const int cmA = warp & 3, h = lane >> 4, q4 = (lane >> 2) & 3;
    const int cmB = 2 * (warp & 1) + h;
    long long wbq[kBU];
    float wscq[kBU];
#pragma unroll
    for (int vb = 0; vb < kBU; ++vb) {
      const int ub = warp + 8 * vb;
      const int q = ((warp >> 1) + 4 * vb) * 4 + q4;
      wbq[vb] = ub < unitsB ? wbase[2 * q] : -1;
      wscq[vb] = (PREC == kFP16S && ub < unitsB && q < Nq) ? wsc[q] : 1.f;
    }
    float2 v[kAppU];
    auto load_chunk = [&](int ch) {
      const int kap0 = ch * KC;
      const int dA = PREC == kTF32X3 ? (kap0 + cmA * 4 + (lane & 3)) >> 1 : (kap0 + cmA * 8 + (lane & 3) * 2) >> 1;
      const int dB = PREC == kTF32X3 ? (kap0 + cmB * 4 + (lane & 3)) >> 1 : (kap0 + cmB * 8 + (lane & 3) * 2) >> 1;
      const long long baseA = dA < D ? colbase[dA] + r0 : -1;
#pragma unroll
      for (int uu = 0; uu < kAU; ++uu) {
        const int row = (warp >> 2) * 8 + 16 * uu + (lane >> 2);
        v[uu] = (baseA >= 0 && r0 + row < R &&
                 in_bounds(baseA + row, ((long long)C * K - 1) * ldr + R, kSiteTcIn))
                    ? __ldg(dop + baseA + row) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int vb = 0; vb < kBU; ++vb) {
        const long long wb = wbq[vb];
        v[kAU + vb] = (dB < D && wb >= 0 && in_bounds(wb + dB, (long long)K * NB * S * D, kSiteTcIn))
                          ? __ldg(wts + wb + dB) : make_float2(0.f, 0.f);
      }
    };
    if (ok) load_chunk(0);
    for (int ch = 0; ch < nchunks && ok; ++ch, ++gch) {
      const int st = (int)(gch & 1);
      uint8_t* stage = sm + st * STAGE;
      if (pending[st]) {
        ok = tc::mbar_wait(&mbar[st], parity[st], wait_polls);
        if (ok) {
          parity[st] ^= 1u;
          pending[st] = false;
        }
      }
      ok = __syncthreads_and(ok);
      if (!ok) break;
      const int kap0 = ch * KC;
#pragma unroll
      for (int uu = 0; uu < kAU; ++uu) {   // A: cell rows
        const float2 e = v[uu];
        const int off = ((warp >> 2) + 2 * uu) * SBO + cmA * 128 + (lane >> 2) * 16 + (lane & 3) * 4;
        if (!in_bounds(off + 3, kAppA, kSiteTcSmem)) continue;   // the word's last byte
        if constexpr (PREC == kTF32X3) {
          const int kap = kap0 + cmA * 4 + (lane & 3);
          uint32_t w[2];
          split_tf32((kap & 1) ? e.y : e.x, w);
          *reinterpret_cast<uint32_t*>(stage + off) = w[0];
          *reinterpret_cast<uint32_t*>(stage + PIECE + off) = w[1];
        } else if constexpr (PREC == kBF16X3) {
          uint32_t w[3];
          split_bf16(e.x, e.y, w);
#pragma unroll
          for (int pc = 0; pc < 3; ++pc) *reinterpret_cast<uint32_t*>(stage + pc * PIECE + off) = w[pc];
        } else {
          uint32_t w[2];
          split_f16(e.x * xsc_s, e.y * xsc_s, w);
          *reinterpret_cast<uint32_t*>(stage + off) = w[0];
          *reinterpret_cast<uint32_t*>(stage + PIECE + off) = w[1];
        }
      }
#pragma unroll
      for (int vb = 0; vb < kBU; ++vb) {   // B: weight rows
        if (warp + 8 * vb >= unitsB) continue;
        const float2 e = v[kAU + vb];
        const int rg = (warp >> 1) + 4 * vb;
        const int offE = kAppA + rg * SBO + cmB * 128 + (2 * q4) * 16 + (lane & 3) * 4;
        const int offO = offE + 16;   // the odd row of the same vector
        if (!in_bounds(offO + 3, PIECE, kSiteTcSmem)) continue;
        // the first store takes even rows in lanes 0-15 and odd rows in
        // lanes 16-31 (and the second the other way round), so each store
        // covers all 32 banks
        const int o1 = h ? offO : offE, o2 = h ? offE : offO;
        constexpr int NPC = F::NPC;
        uint32_t we[NPC], wo[NPC];
        if constexpr (PREC == kTF32X3) {
          // word l & 3 of a row is K element 2 d + (l & 1): even row wr, wi;
          // odd row -wi, wr
          uint32_t pr_[2], pi_[2];
          split_tf32(e.x, pr_);
          split_tf32(e.y, pi_);
          const bool im_word = (lane & 1) != 0;
#pragma unroll
          for (int pc = 0; pc < 2; ++pc) {
            we[pc] = im_word ? pi_[pc] : pr_[pc];
            wo[pc] = im_word ? pr_[pc] : (pi_[pc] ^ 0x80000000u);
          }
        } else {
          // 16-bit pairs (re in the low half): odd word = (-im, re)
          if constexpr (PREC == kBF16X3) {
            split_bf16(e.x, e.y, we);
          } else {
            const float sc = wscq[vb];
            split_f16(e.x * sc, e.y * sc, we);
          }
#pragma unroll
          for (int pc = 0; pc < NPC; ++pc) wo[pc] = ((we[pc] >> 16) ^ 0x8000u) | (we[pc] << 16);
        }
#pragma unroll
        for (int pc = 0; pc < NPC; ++pc) {
          *reinterpret_cast<uint32_t*>(stage + pc * PIECE + o1) = h ? wo[pc] : we[pc];
          *reinterpret_cast<uint32_t*>(stage + pc * PIECE + o2) = h ? we[pc] : wo[pc];
        }
      }
      if (ch + 1 < nchunks) load_chunk(ch + 1);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t base = tc::smem_u32(stage);
#pragma unroll
        for (int ks = 0; ks < KC / F::KI; ++ks) {
          const uint32_t o = ks * 256;
#pragma unroll
          for (int pr = 0; pr < F::NPROD; ++pr) {
            const uint32_t pa = base + prod_a(pr) * PIECE + o;
            const uint32_t pb = base + prod_b(pr) * PIECE + kAppA + o;
            issue_mma<PREC>(tmem, tc::smem_desc(pa, 128, SBO), tc::smem_desc(pb, 128, SBO), idesc,
                            !(ch == 0 && ks == 0 && pr == 0));
          }
        }
        tc::mma_commit(&mbar[st]);
      }
      pending[st] = true;
    }
    for (int s2 = 0; s2 < 2; ++s2) {
      if (pending[s2] && ok) {
        ok = tc::mbar_wait(&mbar[s2], parity[s2], wait_polls);
        if (ok) {
          parity[s2] ^= 1u;
          pending[s2] = false;
        }
      }
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after_sync();
    // epilogue: lane m of warp quarter q4 is cell r0 + m; columns 2 (j S + s)
    // and 2 (j S + s) + 1 hold Re y and Im y of its block j
    {
      const int q4 = warp & 3, hf = warp >> 2;
      const int m = q4 * 32 + lane;
      const int r = r0 + m;
      const bool mine = r < R;
      const int j = mine ? r / B - b0 : -1;
      const int jw0 = (r0 + q4 * 32) / B - b0;
      const int jw1 = min(nbt - 1, (r0 + q4 * 32 + 31) / B - b0);
      const uint32_t lb = (uint32_t)(q4 * 32) << 16;
      for (int jj = jw0; jj <= jw1; ++jj) {
        // blocks of 8 columns starting on a multiple of 8 (column 2 jj S is
        // even, so a (Re, Im) pair never straddles two blocks)
        const int c_lo = 2 * jj * S, c_hi = c_lo + 2 * S;
        for (int cb = (c_lo & ~7) + hf * 8; cb < c_hi; cb += 16) {   // warp-uniform bounds
          float a[8];
          in_bounds(cb + 7, tmem_cols, kSiteTcTmem);   // recorded only
          tc::tmem_ld8(tmem + lb + cb, a);
          if (mine && j == jj) {
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              const int s = (cb + u - c_lo) >> 1;
              if (cb + u >= c_lo && s < S) {
                float re = a[u], im = a[u + 1];
                if constexpr (PREC == kFP16S) {
                  const float inv = winv[jj * S + s];
                  re *= inv;
                  im *= inv;
                }
                if (in_bounds(((long long)s * K + k) * ldr + r, ((long long)S * K - 1) * ldr + R, kSiteTcOut))
                  out[((size_t)s * K + k) * ldr + r] = fmaf(re, re, im * im);
              }
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicExch(&status->timeout, 1u);
    for (int s2 = 0; s2 < 2; ++s2)
      if (pending[s2]) tc::mbar_wait(&mbar[s2], parity[s2], kWaitIter);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

template <int PREC, bool STK>
cudaError_t launch_cov_form(const float2* dop, double2* cov, int C, int K, int R, int ldr, int T, int B,
                            bool lower_only, DeviceStatus* status, cudaStream_t s, int wait_polls) {
  const int D = C * T;
  const int NB = R / B;
  const int D8 = (D + 7) / 8 * 8;
  const int G = CovForm<STK>::GROWS / D8;
  const long long nsys = (long long)K * NB;
  const long long ntiles = (nsys + G - 1) / G;
  const size_t smem = cov_smem<PREC>();
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(covariance_tcx_kernel<PREC, STK>, smem, set_bytes);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM: registers and shared memory (occupancy query),
  // and no more than the SM's 512 TMEM columns hold
  int per_sm = resident_ctas(covariance_tcx_kernel<PREC, STK>, kThreads, smem);
  if (per_sm > 512 / CovForm<STK>::COLS) per_sm = 512 / CovForm<STK>::COLS;
  const long long cap = 152LL * per_sm;
  const long long blocks = ntiles < cap ? ntiles : cap;
  return launch_or_defer(s, [=](cudaStream_t st) {
    covariance_tcx_kernel<PREC, STK><<<(unsigned)blocks, kThreads, smem, st>>>(
        dop, cov, C, K, ldr, T, B, NB, D8, G, ntiles, lower_only ? 1 : 0, status, wait_polls);
    return cudaGetLastError();
  });
}

template <int PREC>
cudaError_t launch_cov(const float2* dop, double2* cov, int C, int K, int R, int ldr, int T, int B,
                       bool lower_only, DeviceStatus* status, cudaStream_t s, int wait_polls) {
  const int D8 = (C * T + 7) / 8 * 8;
  if (D8 <= 64)   // the stacked form: [Xr ; Xi] fill the 128 rows of M
    return launch_cov_form<PREC, true>(dop, cov, C, K, R, ldr, T, B, lower_only, status, s, wait_polls);
  return launch_cov_form<PREC, false>(dop, cov, C, K, R, ldr, T, B, lower_only, status, s, wait_polls);
}

template <int PREC>
cudaError_t launch_app(const float2* dop, const float2* wts, float* out, int C, int K, int R, int ldr,
                       int T, int B, int S, DeviceStatus* status, cudaStream_t s, int wait_polls) {
  const int NB = R / B;
  const int nbt = B < 128 ? 128 / B : 1;
  const int NP = (2 * nbt * S + 15) / 16 * 16;
  // TMEM columns: a power of two >= 32 that holds NP columns plus the
  // epilogue's whole blocks of 8
  int cols = 32;
  while (cols < NP + 8) cols <<= 1;
  const long long ntiles = (long long)K * ((R + 127) / 128);
  const size_t smem = apply_smem<PREC>(NP);
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(apply_tcx_kernel<PREC>, smem, set_bytes);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM: registers and shared memory (occupancy query),
  // and no more than the SM's 512 TMEM columns hold
  int per_sm = resident_ctas(apply_tcx_kernel<PREC>, kThreads, smem);
  if (per_sm > 512 / cols) per_sm = 512 / cols;
  const long long cap = 152LL * per_sm;
  const long long blocks = ntiles < cap ? ntiles : cap;
  return launch_or_defer(s, [=](cudaStream_t st) {
    apply_tcx_kernel<PREC><<<(unsigned)blocks, kThreads, smem, st>>>(dop, wts, out, C, K, R, ldr, T, B, S,
                                                                   NB, NP, cols, ntiles, status,
                                                                   wait_polls);
    return cudaGetLastError();
  });
}

}  // namespace

bool tc_precision(int precision) {
  return precision == STAP_PREC_TF32X3 || precision == STAP_PREC_BF16X3 ||
         precision == STAP_PREC_FP16_SCALED;
}

cudaError_t launch_covariance_tc(const float2* dop, double2* cov, int C, int K, int R, int ldr, int T,
                                 int B, int precision, bool lower_only, DeviceStatus* status,
                                 cudaStream_t s, int wait_polls) {
  if (R / B == 0) return cudaSuccess;
  if (C * T > 128) return cudaErrorInvalidValue;
  switch (precision) {
    case STAP_PREC_TF32X3:
      return launch_cov<kTF32X3>(dop, cov, C, K, R, ldr, T, B, lower_only, status, s, wait_polls);
    case STAP_PREC_BF16X3:
      return launch_cov<kBF16X3>(dop, cov, C, K, R, ldr, T, B, lower_only, status, s, wait_polls);
    case STAP_PREC_FP16_SCALED:
      return launch_cov<kFP16S>(dop, cov, C, K, R, ldr, T, B, lower_only, status, s, wait_polls);
  }
  return cudaErrorInvalidValue;
}

bool apply_tc_supported(int B, int S) {
  const bool tiles = (B <= 128 && 128 % B == 0) || (B % 128 == 0);
  if (!tiles) return false;
  const int nbt = B < 128 ? 128 / B : 1;
  return 2 * nbt * S <= 256;
}

cudaError_t launch_apply_tc(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                            int ldr, int T, int B, int S, int precision, DeviceStatus* status,
                            cudaStream_t s, int wait_polls) {
  if (R / B == 0) return cudaSuccess;
  if (!apply_tc_supported(B, S) || C * T > 128) return cudaErrorInvalidValue;
  switch (precision) {
    case STAP_PREC_TF32X3:
      return launch_app<kTF32X3>(dop, wts, out, C, K, R, ldr, T, B, S, status, s, wait_polls);
    case STAP_PREC_BF16X3:
      return launch_app<kBF16X3>(dop, wts, out, C, K, R, ldr, T, B, S, status, s, wait_polls);
    case STAP_PREC_FP16_SCALED:
      return launch_app<kFP16S>(dop, wts, out, C, K, R, ldr, T, B, S, status, s, wait_polls);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stap

namespace stap {
cudaError_t check_record_mixed(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
