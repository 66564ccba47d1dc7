// Mixed-precision contractions on the tensor cores (tcgen05, kind::tf32).
//
// Covariance per (Doppler bin, range block), R = (1/B) X X^H with X the D x B
// snapshot tile, as three real accumulators in TMEM:
//   Re R = Xr Xr^T + Xi Xi^T,   Im R = Xi Xr^T - Xr Xi^T
// (accumulators A = Xr Xr^T + Xi Xi^T, Bm = Xi Xr^T, Cm = Xr Xi^T; Im R =
// Bm - Cm in the epilogue).  Every product is a 3xTF32 split, hi*hi + hi*lo +
// lo*hi with hi = tf32(v), lo = tf32(v - hi), accumulated in FP32 by the
// tensor core: about 2^-21 relative per product instead of TF32's 2^-11.
// The M = N = 128 tile holds floor(128 / D) systems on its diagonal (rows and
// columns g*D .. g*D + D - 1 belong to system g; off-diagonal blocks are
// never read), so D up to 128 needs no second tile.  Thread i of the CTA owns
// TMEM lane i, i.e. row i of all three accumulators, so the epilogue forms
// its row of R without any exchange.
//
// Pipeline per CTA (128 threads): the B cells are staged in chunks of 32 into
// one of two shared-memory stages (four 128 x 32 TF32 tiles: Xr hi/lo, Xi
// hi/lo, in the K-major core-matrix layout), thread 0 issues the 48 MMAs of
// the chunk and commits them to that stage's mbarrier, and the next chunk is
// staged into the other stage meanwhile.  All waits are bounded: a pipeline
// wait gives up after wait_polls polls (a launch argument, default
// kDefaultWaitPolls); the CTA then records a timeout in the device status,
// waits (bounded by kDefaultWaitPolls) for the MMAs it still has in flight,
// frees its TMEM and stops.  A stage whose wait gave up stays pending, so that
// final drain covers it.
#include "snapshots.cuh"
#include "tcgen05.cuh"

namespace stap {
namespace {

constexpr int kTcThreads = 256;              // 8 warps stage; warps 0-3 own the TMEM lanes
constexpr int kUnroll = 8;                    // staging loads in flight per lane
constexpr int kKC = 32;                       // cells per chunk (K of one stage)
constexpr int kTile = 128 * kKC * 4;          // one 128 x 32 TF32 operand tile (16 KB)
constexpr int kStage = 4 * kTile;             // Xr hi, Xr lo, Xi hi, Xi lo (64 KB)
constexpr int kWaitIter = kDefaultWaitPolls;    // drain waits before TMEM is freed
constexpr int kTmemCols = 512;                // 3 x 128 accumulators, rounded up

__global__ void __launch_bounds__(kTcThreads)
covariance_tc_kernel(const float2* __restrict__ dop, double2* __restrict__ cov, int C, int K,
                     int ldr, int T, int B, int NB, int G, long long ntiles,
                     DeviceStatus* __restrict__ status, int wait_polls) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ long long rowbase[128];          // dop offset of each tile row's range block, or -1
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = C * T;
  const int rows = G * D;
  const long long nsys = (long long)K * NB;
  const int nchunks = (B + kKC - 1) / kKC;

  for (int i = tid; i < 2 * kStage / 4; i += kTcThreads) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t accA = tmem, accB = tmem + 128, accC = tmem + 256;
  const uint32_t idesc = tc::idesc_tf32(128, 128);
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  long long gch = 0;                          // chunks issued by this CTA (stage = gch & 1)

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long sys0 = tile * G;
    if (tid < 128) {  // row p = g*D + i: snapshot entry i of system sys0 + g
      long long base = -1;
      if (tid < rows) {
        const int g = tid / D, i = tid - g * D;
        const long long sys = sys0 + g;
        if (sys < nsys) {
          const int k = (int)(sys / NB), b = (int)(sys - (long long)k * NB);
          const int t = i / C, c = i - t * C;
          const int kk = wrap_bin(k + t - T / 2, K);
          base = ((long long)c * K + kk) * ldr + (long long)b * B;
        }
      }
      rowbase[tid] = base;
    }
    for (int ch = 0; ch < nchunks && ok; ++ch, ++gch) {
      const int st = (int)(gch & 1);
      uint8_t* stage = sm + st * kStage;
      if (pending[st]) {  // the MMAs that last read this stage must be done
        ok = tc::mbar_wait(&mbar[st], parity[st], wait_polls);
        if (ok) {
          parity[st] ^= 1u;
          pending[st] = false;
        }
      }
      ok = __syncthreads_and(ok);
      if (!ok) break;
      // stage cells c0 .. c0+31: one core matrix (8 rows x 4 cells) per warp
      // pass, kUnroll loads in flight per lane before the conversions
      const int c0 = ch * kKC;
      const int ncm = (rows + 7) / 8 * (kKC / 4);
      constexpr int NWS = kTcThreads / 32;
      for (int cb0 = warp; cb0 < ncm; cb0 += NWS * kUnroll) {
        float2 xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int cmi = cb0 + u * NWS;
          xv[u] = make_float2(0.f, 0.f);
          if (cmi < ncm) {
            const int p = (cmi >> 3) * 8 + (lane >> 2), j = (cmi & 7) * 4 + (lane & 3);
            const long long base = rowbase[p];
            if (base >= 0 && c0 + j < B) xv[u] = __ldg(dop + base + c0 + j);
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int cmi = cb0 + u * NWS;
          if (cmi < ncm) {
            const int p = (cmi >> 3) * 8 + (lane >> 2), j = (cmi & 7) * 4 + (lane & 3);
            const float2 x = xv[u];
            const uint32_t rh = tc::to_tf32(x.x), ih = tc::to_tf32(x.y);
            const uint32_t rl = tc::to_tf32(x.x - __uint_as_float(rh));
            const uint32_t il = tc::to_tf32(x.y - __uint_as_float(ih));
            const int off = tc::cm_offset(p, j, kKC);
            *reinterpret_cast<uint32_t*>(stage + 0 * kTile + off) = rh;
            *reinterpret_cast<uint32_t*>(stage + 1 * kTile + off) = rl;
            *reinterpret_cast<uint32_t*>(stage + 2 * kTile + off) = ih;
            *reinterpret_cast<uint32_t*>(stage + 3 * kTile + off) = il;
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t base = tc::smem_u32(stage);
        const uint32_t rh = base, rl = base + kTile, ih = base + 2 * kTile, il = base + 3 * kTile;
        constexpr uint32_t LBO = 128, SBO = 128 * (kKC / 4);
        for (int ks = 0; ks < kKC / 8; ++ks) {
          const uint32_t o = ks * 256;
          const bool first = (ch == 0 && ks == 0);
          const uint64_t drh = tc::smem_desc(rh + o, LBO, SBO), drl = tc::smem_desc(rl + o, LBO, SBO);
          const uint64_t dih = tc::smem_desc(ih + o, LBO, SBO), dil = tc::smem_desc(il + o, LBO, SBO);
          // A += Xr Xr^T + Xi Xi^T
          tc::mma_tf32(accA, drh, drh, idesc, !first);
          tc::mma_tf32(accA, drh, drl, idesc, true);
          tc::mma_tf32(accA, drl, drh, idesc, true);
          tc::mma_tf32(accA, dih, dih, idesc, true);
          tc::mma_tf32(accA, dih, dil, idesc, true);
          tc::mma_tf32(accA, dil, dih, idesc, true);
          // Bm += Xi Xr^T
          tc::mma_tf32(accB, dih, drh, idesc, !first);
          tc::mma_tf32(accB, dih, drl, idesc, true);
          tc::mma_tf32(accB, dil, drh, idesc, true);
          // Cm += Xr Xi^T
          tc::mma_tf32(accC, drh, dih, idesc, !first);
          tc::mma_tf32(accC, drh, dil, idesc, true);
          tc::mma_tf32(accC, drl, dih, idesc, true);
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
    // epilogue (warps 0-3): thread tid owns row tid of the tile = row i of system g
    const int g = tid / D, i = tid - g * D;
    const long long sys = sys0 + g;
    const bool mine = tid < 128 && tid < rows && sys < nsys;
    const float invBf = 1.0f / (float)B;
    double2* out = cov + (size_t)(mine ? sys : 0) * D * D;
    const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
    for (int cb = 0; cb < rows && warp < 4; cb += 8) {   // columns in blocks of 8 (warp-collective)
      float a[8], bm[8], cm[8];
      tc::tmem_ld8(accA + lanebase + cb, a);
      tc::tmem_ld8(accB + lanebase + cb, bm);
      tc::tmem_ld8(accC + lanebase + cb, cm);
      if (mine) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int col = cb + u;
          const int l = col - g * D;
          if (l >= 0 && l <= i && l < D) {        // lower triangle of this system, mirrored
            const double re = (double)(a[u] * invBf);
            const double im = (l == i) ? 0.0 : (double)((bm[u] - cm[u]) * invBf);
            out[(size_t)i * D + l] = make_double2(re, im);
            if (l != i) out[(size_t)l * D + i] = make_double2(re, -im);
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM reads done before the next tile's MMAs overwrite it
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicExch(&status->timeout, 1u);
    for (int s2 = 0; s2 < 2; ++s2)      // let MMAs still in flight finish (bounded)
      if (pending[s2]) tc::mbar_wait(&mbar[s2], parity[s2], kWaitIter);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Apply, out[s][k][r] = |w_{k,b(r),s}^H x_{k,r}|^2, as a real GEMM per tile of
// 128 range cells of one Doppler bin (M = cells, N = steering vectors of the
// nbt blocks the tile covers, K = D):
//   Re y = Xr Wr^T + Xi Wi^T,   Im y = Xi Wr^T - Xr Wi^T
// with accumulators A = Xr Wr^T + Xi Wi^T, Bm = Xi Wr^T, Cm = Xr Wi^T, each a
// 3xTF32 product.  Column j*S + s of the tile holds steering vector s of the
// tile's block j; a cell only reads its own block's columns.  K = D goes in
// double-buffered chunks of 16.  Thread m owns TMEM lane m (cell r0 + m), so
// the epilogue writes each output row out[s][k][r0 .. r0+127] coalesced.
constexpr int kAKC = 16;                      // snapshot entries per chunk
constexpr int kAX = 128 * kAKC * 4;           // one 128 x 16 TF32 tile (8 KB)
constexpr int kAStage = 8 * kAX;              // X: re/im x hi/lo, W: re/im x hi/lo (64 KB)

__global__ void __launch_bounds__(kTcThreads)
apply_tc_kernel(const float2* __restrict__ dop, const float2* __restrict__ wts,
                float* __restrict__ out, int C, int K, int R, int ldr, int T, int B, int S, int NB,
                int NP, long long ntiles, DeviceStatus* __restrict__ status,
                int wait_polls) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ long long colbase[128];          // dop offset of snapshot entry d's row (bin k)
  __shared__ long long wbase[128];            // wts offset of weight row n, or -1
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int D = C * T;
  const int tiles_per_k = (R + 127) / 128;
  const int nbt_max = B < 128 ? 128 / B : 1;
  const int N = nbt_max * S;
  const int nchunks = (D + kAKC - 1) / kAKC;

  for (int i = tid; i < 2 * kAStage / 4; i += kTcThreads) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t accA = tmem, accB = tmem + 128, accC = tmem + 256;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  long long gch = 0;

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int k = (int)(tile / tiles_per_k);
    const int r0 = (int)(tile - (long long)k * tiles_per_k) * 128;
    const int b0 = r0 / B;
    if (tid < 128) {
      if (tid < D) {
        const int t = tid / C, c = tid - t * C;
        colbase[tid] = ((long long)c * K + wrap_bin(k + t - T / 2, K)) * ldr;
      }
      const int j = tid / S, s = tid - j * S;
      wbase[tid] = (tid < N && b0 + j < NB) ? ((((long long)k * NB + b0 + j) * S + s) * D) : -1;
    }
    for (int ch = 0; ch < nchunks && ok; ++ch, ++gch) {
      const int st = (int)(gch & 1);
      uint8_t* stage = sm + st * kAStage;
      if (pending[st]) {
        ok = tc::mbar_wait(&mbar[st], parity[st], wait_polls);
        if (ok) {
          parity[st] ^= 1u;
          pending[st] = false;
        }
      }
      ok = __syncthreads_and(ok);
      if (!ok) break;
      const int d0 = ch * kAKC;
      // X tile (rows = cells) and W tile (rows n = j*S + s of block b0 + j),
      // K = snapshot entries d0 .. d0+15; kUnroll loads in flight per lane
      constexpr int NWS = kTcThreads / 32;
      const int ncx = 16 * (kAKC / 4), ncw = (NP / 8) * (kAKC / 4), ncm = ncx + ncw;
      for (int cb0 = warp; cb0 < ncm; cb0 += NWS * kUnroll) {
        float2 xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int cmi = cb0 + u * NWS;
          xv[u] = make_float2(0.f, 0.f);
          if (cmi < ncx) {
            const int m = (cmi >> 2) * 8 + (lane >> 2), d = d0 + (cmi & 3) * 4 + (lane & 3);
            const int r = r0 + m;
            if (d < D && r < R) xv[u] = __ldg(dop + colbase[d] + r);
          } else if (cmi < ncm) {
            const int cw = cmi - ncx;
            const int n = (cw >> 2) * 8 + (lane >> 2), d = d0 + (cw & 3) * 4 + (lane & 3);
            const long long wb = wbase[n];
            if (wb >= 0 && d < D) xv[u] = __ldg(wts + wb + d);
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int cmi = cb0 + u * NWS;
          if (cmi < ncm) {
            const bool isx = cmi < ncx;
            const int cl = isx ? cmi : cmi - ncx;
            const int row = (cl >> 2) * 8 + (lane >> 2), dd = (cl & 3) * 4 + (lane & 3);
            const float2 x = xv[u];
            const uint32_t rh = tc::to_tf32(x.x), ih = tc::to_tf32(x.y);
            const uint32_t rl = tc::to_tf32(x.x - __uint_as_float(rh));
            const uint32_t il = tc::to_tf32(x.y - __uint_as_float(ih));
            uint8_t* t0 = stage + (isx ? 0 : 4 * kAX) + tc::cm_offset(row, dd, kAKC);
            *reinterpret_cast<uint32_t*>(t0 + 0 * kAX) = rh;
            *reinterpret_cast<uint32_t*>(t0 + 1 * kAX) = rl;
            *reinterpret_cast<uint32_t*>(t0 + 2 * kAX) = ih;
            *reinterpret_cast<uint32_t*>(t0 + 3 * kAX) = il;
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t base = tc::smem_u32(stage);
        constexpr uint32_t LBO = 128, SBO = 128 * (kAKC / 4);
        for (int ks = 0; ks < kAKC / 8; ++ks) {
          const uint32_t o = ks * 256;
          const bool first = (ch == 0 && ks == 0);
          const uint64_t xrh = tc::smem_desc(base + 0 * kAX + o, LBO, SBO);
          const uint64_t xrl = tc::smem_desc(base + 1 * kAX + o, LBO, SBO);
          const uint64_t xih = tc::smem_desc(base + 2 * kAX + o, LBO, SBO);
          const uint64_t xil = tc::smem_desc(base + 3 * kAX + o, LBO, SBO);
          const uint64_t wrh = tc::smem_desc(base + 4 * kAX + o, LBO, SBO);
          const uint64_t wrl = tc::smem_desc(base + 5 * kAX + o, LBO, SBO);
          const uint64_t wih = tc::smem_desc(base + 6 * kAX + o, LBO, SBO);
          const uint64_t wil = tc::smem_desc(base + 7 * kAX + o, LBO, SBO);
          // A += Xr Wr^T + Xi Wi^T
          tc::mma_tf32(accA, xrh, wrh, idesc, !first);
          tc::mma_tf32(accA, xrh, wrl, idesc, true);
          tc::mma_tf32(accA, xrl, wrh, idesc, true);
          tc::mma_tf32(accA, xih, wih, idesc, true);
          tc::mma_tf32(accA, xih, wil, idesc, true);
          tc::mma_tf32(accA, xil, wih, idesc, true);
          // Bm += Xi Wr^T
          tc::mma_tf32(accB, xih, wrh, idesc, !first);
          tc::mma_tf32(accB, xih, wrl, idesc, true);
          tc::mma_tf32(accB, xil, wrh, idesc, true);
          // Cm += Xr Wi^T
          tc::mma_tf32(accC, xrh, wih, idesc, !first);
          tc::mma_tf32(accC, xrh, wil, idesc, true);
          tc::mma_tf32(accC, xrl, wih, idesc, true);
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
    // epilogue (warps 0-3): cell r0 + tid, block b0 + j, columns j*S .. j*S + S - 1
    const int r = r0 + tid;
    const int j = (r / B) - b0;
    const bool mine = tid < 128 && r < R;
    const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
    for (int cb = 0; cb < NP && warp < 4; cb += 8) {
      float a[8], bm[8], cm[8];
      tc::tmem_ld8(accA + lanebase + cb, a);
      tc::tmem_ld8(accB + lanebase + cb, bm);
      tc::tmem_ld8(accC + lanebase + cb, cm);
      if (mine) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int s = cb + u - j * S;
          if (s >= 0 && s < S) {
            const float re = a[u], im = bm[u] - cm[u];
            out[((size_t)s * K + k) * ldr + r] = fmaf(re, re, im * im);
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
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

cudaError_t launch_covariance_tc(const float2* dop, double2* cov, int C, int K, int R, int ldr, int T,
                                 int B, DeviceStatus* status, cudaStream_t s, int wait_polls) {
  const int D = C * T;
  const int NB = R / B;
  if (NB == 0) return cudaSuccess;
  if (D > 128) return cudaErrorInvalidValue;
  const int G = 128 / D;
  const long long nsys = (long long)K * NB;
  const long long ntiles = (nsys + G - 1) / G;
  const size_t smem = 2 * (size_t)kStage;
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(covariance_tc_kernel, smem, set_bytes);
  if (e != cudaSuccess) return e;
  long long blocks = ntiles < 152 ? ntiles : 152;   // one CTA per SM (TMEM and shared memory)
  covariance_tc_kernel<<<(unsigned)blocks, kTcThreads, smem, s>>>(dop, cov, C, K, ldr, T, B, NB, G,
                                                                    ntiles, status,
                                                                    wait_polls);
  return cudaGetLastError();
}

bool apply_tc_supported(int B, int S) {
  const bool tiles = (B <= 128 && 128 % B == 0) || (B % 128 == 0);
  if (!tiles) return false;
  const int N = (B < 128 ? 128 / B : 1) * S;
  return (N + 15) / 16 * 16 <= 128;
}

cudaError_t launch_apply_tc(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                            int ldr, int T, int B, int S, DeviceStatus* status, cudaStream_t s,
                            int wait_polls) {
  const int NB = R / B;
  if (NB == 0) return cudaSuccess;
  if (!apply_tc_supported(B, S) || C * T > 128) return cudaErrorInvalidValue;
  const int N = (B < 128 ? 128 / B : 1) * S;
  const int NP = (N + 15) / 16 * 16;
  const long long ntiles = (long long)K * ((R + 127) / 128);
  const size_t smem = 2 * (size_t)kAStage;
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(apply_tc_kernel, smem, set_bytes);
  if (e != cudaSuccess) return e;
  long long blocks = ntiles < 152 ? ntiles : 152;
  apply_tc_kernel<<<(unsigned)blocks, kTcThreads, smem, s>>>(dop, wts, out, C, K, R, ldr, T, B, S, NB, NP,
                                                               ntiles, status, wait_polls);
  return cudaGetLastError();
}

}  // namespace stap
