// Internal declarations of libstap: kernel launchers, the device status block
// and small complex helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "stap.h"

namespace stap {

// Device-side status, at offset 0 of the workspace.
struct DeviceStatus {
  unsigned long long n_failed;   // systems whose loaded covariance was not positive definite
  unsigned int timeout;          // a bounded wait gave up (1)
  unsigned int pad[13];
};
static_assert(sizeof(DeviceStatus) <= 256, "status block must fit its slot");

constexpr int kMaxD = 128;       // largest snapshot length the solve kernels handle
constexpr int kSmallMaxD = 32;   // above this, one system per CTA (lanes over rows)
constexpr int kMaxLogK = 10;     // K <= 1024
constexpr int kDefaultWaitPolls = STAP_DEFAULT_WAIT_POLLS;   // mbarrier polls before a bounded wait gives up

// Launch choices the autotuner can make for one CPI shape (0 = the built-in
// heuristic).  Every choice computes the same result, except that the two FP32
// apply kernels accumulate in a different order.
struct Tune {
  int dop_tr = 0;      // range cells per Doppler CTA: 8, 16 or 32
  int cov_kt = 0;      // Doppler bins per covariance CTA (bin-pair kernel), a divisor of K
  int solve_ts = 0;    // D <= 32 solve: lanes per system (power of two, >= one per RHS)
  int solve_nw = 0;    // D <= 32 solve: warps per CTA, 1..4; D > 64 FP64 solve: 16 for 512-thread CTAs
  int solve_lr = 0;    // D > 32 solve: lanes per right-hand side, 8 (D <= 64), 16 or 32
  int apply_kind = 0;  // apply: 1 FP32 register-resident, 2 FP32 general, 3 tensor cores
  int slabs = 0;       // single-CPI run: range slabs pipelined on prioritised streams, 1..8
  int solve_kind = 0;  // D <= 32 solve: 1 register-resident (D = 8, 12, 16), 2 shared-memory
                       // teams, 3 one system per CTA
  int cov_kind = 0;    // covariance: 1 FP32 error-free, 2 tensor cores (mixed-precision plans)
};

// The FP64 pivot reciprocal of the one-system-per-CTA factorisation on n
// device doubles (test support).
cudaError_t launch_pivot_reciprocal(const double* in, double* out, long long n, cudaStream_t s);

// Training with guard cells: out[k][b] = mean of in[k][b-1] and in[k][b+1]
// (the one that exists at either end); NB >= 2.
cudaError_t launch_train_neighbours(const double2* in, double2* out, int K, int NB, int D,
                                    cudaStream_t s);

// Sliding training window: out[k][j] = mean of in[k][i] over the groups
// i = j-guard-half .. j-guard-1 and j+guard+1 .. j+guard+half in 0 .. NB-1;
// needs guard >= 0, half >= 1, NB >= 2 guard + 2.
cudaError_t launch_train_window(const double2* in, double2* out, int K, int NB, int D, int guard,
                                int half, cudaStream_t s);

// First out-of-range index found by the checked build in one source file
// (checked.cuh): how many accesses were skipped, and the first one's site
// code, index and the extent it was checked against.
struct CheckRecord {
  unsigned long long count;
  long long index;
  long long extent;
  int site;
  int pad;
};
// Each kernel source file's record, read and cleared (zeros in the normal build).
cudaError_t check_record_doppler(CheckRecord* out);
cudaError_t check_record_covariance(CheckRecord* out);
cudaError_t check_record_solve(CheckRecord* out);
cudaError_t check_record_apply(CheckRecord* out);
cudaError_t check_record_mixed(CheckRecord* out);
cudaError_t check_record_train(CheckRecord* out);

// Snapshot lengths with a mixed-precision iterative-refinement solve.
bool mir_supported(int D);

// ---------------------------------------------------------------- launchers --
// Each returns cudaGetLastError() after its launches.

// Hann-windowed DFT over pulses via a two-pass in-register FFT.
// cube [C][P][R] c64 -> dop [C][K][R] c64; win[P] float; tw[K] = exp(-2 pi i m/K).
// Reduced-DOF front end: y[c][p][r] (+)= sum_{n<Nc} conj(W[c][n0+n]) x_chunk[n][p][r]
// for one chunk of Nc element channels (x_chunk [Nc][P][R], W [C][N], y [C][P][R],
// all c64); accumulate adds to y instead of writing it.
cudaError_t launch_reduce_channels(const float2* x_chunk, const float2* W, float2* y, int N, int n0,
                                   int Nc, int C, int P, int R, bool accumulate, cudaStream_t s);

// TW = 1: the plain transform (win: Hann of length P); TW > 1: PRI-staggered
// sub-windows (win: Hann of length P - TW + 1), dop rows t*C + c.
cudaError_t launch_doppler(const float2* cube, float2* dop, const float* win, const float2* tw,
                           int C, int TW, int P, int K, int R, int ldr, cudaStream_t s,
                           const Tune& t = Tune());

// Covariance per (k, block) from the Doppler cube, accumulated error-free in
// FP32 pairs; written as FP64 complex [K][NB][D][D] (full Hermitian).
cudaError_t launch_covariance_fp32(const float2* dop, double2* cov, int C, int K, int R, int ldr,
                                   int T, int B, cudaStream_t s, const Tune& t = Tune());

// True for the precisions whose covariance and apply run on the tensor cores.
bool tc_precision(int precision);

// The same covariance from split tensor-core products (tcgen05) with FP32
// accumulation, in the arithmetic of `precision` (STAP_PREC_TF32X3,
// STAP_PREC_BF16X3 or STAP_PREC_FP16_SCALED).  lower_only: write only the
// lower triangle (with the real diagonal) of each system, which is all the
// solve reads; otherwise the full Hermitian matrix.  wait_polls: polls before
// a pipeline wait gives up (kDefaultWaitPolls normally).
cudaError_t launch_covariance_tc(const float2* dop, double2* cov, int C, int K, int R, int ldr, int T,
                                 int B, int precision, bool lower_only, DeviceStatus* status,
                                 cudaStream_t s, int wait_polls = kDefaultWaitPolls);

// Apply from split tensor-core products; needs B | 128 or 128 | B and at most
// 256 real weight rows (two per steering vector and block) per 128-cell tile
// (apply_tc_supported).
bool apply_tc_supported(int B, int S);
cudaError_t launch_apply_tc(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                            int ldr, int T, int B, int S, int precision, DeviceStatus* status,
                            cudaStream_t s, int wait_polls = kDefaultWaitPolls);

// FP64 loading, Cholesky, solves, refinement and scaling for nsys systems.
// cov [nsys][D][D] c128 -> wts [nsys][S][D] c64; steer [S][D] c128.  If
// sep_g [T] and sep_a [S][C] are given, steer[s] = sep_g (x) sep_a[s] and the
// solve runs on the C basis vectors instead of the S steering vectors.
// steer_ff [S][D] and sep_a_ff [S][C] are the same tables as double-floats
// (re_hi, re_lo, im_hi, im_lo) for the combination on the FP32 pipe.
cudaError_t launch_solve(const double2* cov, float2* wts, const double2* steer,
                         const double2* sep_g, const double2* sep_a, const float4* steer_ff,
                         const float4* sep_a_ff, const float4* g_ff, long long nsys, int D, int S,
                         int C, double load_factor, int refine_steps, int solver,
                         DeviceStatus* status, cudaStream_t s, const Tune& t = Tune(),
                         bool sep_sym = false);

// out[s][k][r] = |w^H x|^2; dop [C][K][R] c64, wts [K][NB][S][D] c64, out [S][K][R] f32.
cudaError_t launch_apply(const float2* dop, const float2* wts, float* out, int C, int K, int R,
                         int ldr, int T, int B, int S, cudaStream_t s, const Tune& t = Tune());

// ------------------------------------------------------------ device helpers --

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int wrap_bin(int k, int K) {
  int m = k % K;
  return m < 0 ? m + K : m;
}

}  // namespace stap
