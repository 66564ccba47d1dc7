// Adaptive weights per (Doppler bin, range block), all in FP64:
//   delta = lf * Re tr(R) / D,   Rl = R + delta I = L L^H      (diagonal load, Cholesky)
//   u_s = Rl^{-1} v_s            (forward then back substitution)
//   u_s += Rl^{-1} (v_s - Rl u_s)   refine_steps times (residual in FP64 from Rl itself)
//   w_s = u_s / sqrt(Re v_s^H u_s)  (unit noise gain)
// This is the solve half of the STAP kernel of arXiv 2203.06233 Sec. 4.2 (the
// paper gives no formulas; this is the standard loaded-sample-matrix reading).
//
// Cost model on GB300: FP64 FMA runs at 1/62 of the FP32 rate (1.2 TFLOP/s per
// GPU measured), and a warp-wide DFMA costs the same whether 1 or 32 lanes are
// active.  So the kernel is designed around the count of warp-level FP64
// instructions: every lane of every DFMA does useful work, and everything else
// (shared-memory traffic, index arithmetic) is free by comparison.
//
// Mapping: a warp handles G systems at once, TS = 32/G lanes ("a team") per
// system.  The team factors its system right-looking in shared memory (packed
// lower triangle), spreading each trailing update over its lanes, then each
// lane solves for its own right-hand sides (one steering vector per lane and
// pass), reading L as a broadcast and keeping its two work vectors in shared
// memory.  Teams of one warp share all control flow (same D and S), so the
// warp never diverges except where S is not a multiple of TS.
//
// Separable steering (SEP): when every steering vector is v_s = g (x) a_s
// (one temporal factor g of length T shared by all s, a spatial factor a_s of
// length C), Rl^{-1} v_s = sum_c a_s[c] Rl^{-1} (g (x) e_c).  The team then
// solves (and refines) only the C basis right-hand sides g (x) e_c, one per
// lane, and forms each u_s as that FP64 combination, followed by the same
// normalisation.  Exact in exact arithmetic; it cuts the substitution work
// from S to C right-hand sides.  The combination stays in FP64: u_s can be
// two orders of magnitude smaller than the terms it sums (steering vectors
// near the clutter ridge), so FP32 there costs ~1e-4 in the weights.
#include <type_traits>

#include "df64.cuh"
#include "batch.cuh"
#include "checked.cuh"
#include "snapshots.cuh"

namespace stap {
namespace {

__device__ __forceinline__ int pidx(int i, int l) { return i * (i + 1) / 2 + l; }

// Per-team strides of the refinement kernel's shared-memory arrays, rounded
// up to an odd number of elements: the 32 / TS teams of a warp then read the
// same offset of their own arrays from distinct banks.  (Dp = D (D + 1) / 2
// is even for D = 8, 12 and 16: entries at an even stride put two, four or
// eight teams on the same banks.  The FP64 kernels keep the even strides:
// bound by the FP64 pipe, they measured no faster with odd ones.)
__host__ __device__ constexpr int odd_up(int n) { return n | 1; }

// acc -= a * b
__device__ __forceinline__ void cfms(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// acc -= conj(a) * b
__device__ __forceinline__ void cfms_conj(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// acc -= d * b for a real d (a diagonal entry of the loaded matrix)
__device__ __forceinline__ void diag_fms(double2& acc, double d, double2 b) {
  acc.x = fma(-d, b.x, acc.x);
  acc.y = fma(-d, b.y, acc.y);
}

// Lower-triangle element (i, l) of the loaded matrix Rl, i >= l, from the
// full input (only the lower triangle and the real diagonal are read).
__device__ __forceinline__ double2 loaded(const double2* __restrict__ A, int D, int i, int l,
                                          double delta) {
  double2 a = __ldg(A + (size_t)i * D + l);
  if (i == l) {
    a.x += delta;
    a.y = 0.0;
  }
  return a;
}

// x <- (L L^H)^{-1} x in place, x[d] at vec[d * 32] (this lane's column).
__device__ __forceinline__ void chol_solve_inplace(const double2* __restrict__ L,
                                                   const double* __restrict__ invd, double2* vec,
                                                   int D) {
  for (int i = 0; i < D; ++i) {
    double2 acc = vec[i * 32];
    const double2* Li = L + pidx(i, 0);
    for (int l = 0; l < i; ++l) cfms(acc, Li[l], vec[l * 32]);
    const double s = invd[i];
    vec[i * 32] = make_double2(acc.x * s, acc.y * s);
  }
  for (int i = D - 1; i >= 0; --i) {
    double2 acc = vec[i * 32];
    for (int l = i + 1; l < D; ++l) cfms_conj(acc, L[pidx(l, i)], vec[l * 32]);
    const double s = invd[i];
    vec[i * 32] = make_double2(acc.x * s, acc.y * s);
  }
}

// Step the packed lower-triangle coordinates (i, l), l <= i, of index q to
// those of q + step (no division).
__device__ __forceinline__ void step_lower(int& i, int& l, int step) {
  l += step;
  while (l > i) {
    l -= i + 1;
    ++i;
  }
}

// 1/d for a positive, finite, normal d: Newton-Raphson iteration for the
// reciprocal, r <- r + r (1 - d r), whose relative error squares at each step
// (Muller et al., Handbook of Floating-Point Arithmetic, 2nd ed., sec. 4.7),
// started from the hardware's approximate reciprocal; three steps take any
// start error below 2^-8 under FP64's unit roundoff.  The chain of dependent
// FP64 operations is shorter than a full IEEE division's, and in the
// one-system-per-CTA factorisation it sits between two barriers, where each
// of its operations waits behind the other warps' DFMAs in the FP64 pipe.
__device__ __forceinline__ double recip_newton(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
#pragma unroll
  for (int k = 0; k < 3; ++k) r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// (re, im) as the double-floats (re_hi, re_lo, im_hi, im_lo); the split runs
// on the integer pipe, off the FP64 pipe that the FP64 solve kernels are bound by
__device__ __forceinline__ float4 to_ff4(double2 u) {
  const ff::F2 re = ff::from_double(u.x), im = ff::from_double(u.y);
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// the same with the conversion instructions, for the refinement kernels, whose
// FP32 and integer issue is the bottleneck
__device__ __forceinline__ float4 to_ff4_cvt(double2 u) {
  const ff::F2 re = ff::from_double_cvt(u.x), im = ff::from_double_cvt(u.y);
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Separable steering, after the basis solves: u_s = sum_c a_s[c] U_c and
// w_s = u_s / sqrt(Re v_s^H u_s) for the S steering vectors, lane tl of the
// team taking s = tl, tl + TS, ...  The combination and the normalisation are
// not triangular solves; they run in double-float on the FP32 pipe (about
// 2^-48 relative) from the FP64 basis solutions, which Wt holds as
// Wt[i * 32 + c] = to_ff4(U_c[i]).  w: the system's weights [S][D] (nullptr:
// compute nothing to store).
__device__ __forceinline__ void sep_emit(const float4* Wt, int D, int S, int C, int TS, int tl,
                                         const float4* __restrict__ steer_ff,
                                         const float4* __restrict__ sep_a_ff, bool ok,
                                         float2* __restrict__ w) {
  auto combine = [&](int s, int i, ff::F2& ur, ff::F2& ui) {
    const float4* as = sep_a_ff + (size_t)s * C;
    ur = {0.f, 0.f};
    ui = {0.f, 0.f};
    for (int c = 0; c < C; ++c) {
      const float4 a = __ldg(as + c), x = Wt[i * 32 + c];
      const ff::F2 ar{a.x, a.y}, ai{a.z, a.w}, xr{x.x, x.y}, xi{x.z, x.w};
      ur = ff::fms(ff::fma(ur, ar, xr), ai, xi);
      ui = ff::fma(ff::fma(ui, ar, xi), ai, xr);
    }
  };
  // one combination pass: u_s rounded to FP32 goes straight to the weights
  // (the value the scaling multiplies), then a pass over them scales by
  // 1/sqrt(Re v^H u) once that is known
  for (int s0 = 0; s0 < S; s0 += TS) {
    const int s = s0 + tl;
    if (s < S) {
      const float4* v = steer_ff + (size_t)s * D;
      float2* ws = w ? w + (size_t)s * D : nullptr;
      ff::F2 q{0.f, 0.f};                   // Re v^H u
      for (int i = 0; i < D; ++i) {
        ff::F2 ur, ui;
        combine(s, i, ur, ui);
        const float4 vi = __ldg(v + i);
        q = ff::fma(ff::fma(q, {vi.x, vi.y}, ur), {vi.z, vi.w}, ui);
        if (ws) ws[i] = make_float2(__fadd_rn(ur.hi, ur.lo), __fadd_rn(ui.hi, ui.lo));
      }
      const double qd = ff::to_double(q);
      const bool good = ok && qd > 0.0 && isfinite(qd);
      const float sf = good ? (float)rsqrt(qd) : 0.f;
      if (ws)
        for (int i = 0; i < D; ++i) {
          const float2 u = ws[i];
          ws[i] = good ? make_float2(u.x * sf, u.y * sf) : make_float2(0.f, 0.f);
        }
    }
  }
}

// Parameters of one solve launch (one CPI); gx = the launch's grid size.
struct SolveParams {
  const double2* cov;
  float2* wts;
  const double2* steer;
  const double2* sep_g;
  const double2* sep_a;
  const float4* steer_ff;
  const float4* sep_a_ff;
  long long nsys;
  int D, S, C, TS;
  double load_factor;
  int refine_steps;
  DeviceStatus* status;
  int gx;
  int sym;   // the separable spatial factors are conjugate-symmetric: a_{S-1-s} = conj(a_s)
};

template <bool SEP>
__device__ __forceinline__ void solve_kernel_body(const SolveParams& prm, long long bx, long long gx) {
  const double2* __restrict__ cov = prm.cov;
  float2* __restrict__ wts = prm.wts;
  const double2* __restrict__ steer = prm.steer;
  const double2* __restrict__ sep_g = prm.sep_g;
  const float4* __restrict__ steer_ff = prm.steer_ff;
  const float4* __restrict__ sep_a_ff = prm.sep_a_ff;
  const long long nsys = prm.nsys;
  const int S = prm.S, C = prm.C;
  const double load_factor = prm.load_factor;
  const int refine_steps = prm.refine_steps;
  DeviceStatus* __restrict__ status = prm.status;
  (void)steer; (void)sep_g; (void)steer_ff; (void)sep_a_ff;
  const double2* __restrict__ sep_a = prm.sep_a;
  const int D = prm.D, TS = prm.TS;
  (void)sep_a;
  extern __shared__ double2 sm[];
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = 32 / TS, team = lane / TS, tl = lane - team * TS;
  const int Dp = D * (D + 1) / 2;
  const size_t warp_elems = (size_t)G * Dp + 2 * (size_t)D * 32;
  double2* wbase = sm + warp * warp_elems;
  double2* L = wbase + (size_t)team * Dp;          // packed lower factor of this team's system
  double2* U = wbase + (size_t)G * Dp + lane;      // u (this lane's column), stride 32
  double2* W = U + (size_t)D * 32;                 // work vector, stride 32
  double* invd = reinterpret_cast<double*>(sm + nw * warp_elems) + ((size_t)warp * G + team) * D;
  const double invD = 1.0 / (double)D;

  for (long long base = ((long long)bx * nw + warp) * G; base < nsys;
       base += (long long)gx * nw * G) {
    const long long sys = base + team;
    const bool valid = sys < nsys;
    const double2* A = cov + (size_t)(valid ? sys : nsys - 1) * D * D;

    // ---- diagonal load and packed copy of Rl (lower triangle) ----
    double tr = 0.0;
    for (int j = 0; j < D; ++j) tr += __ldg(&A[(size_t)j * D + j].x);
    const double delta = load_factor * tr * invD;
    {
      int i = 0, l = 0;
      step_lower(i, l, tl);
      for (int q = tl; q < Dp; q += TS) {
        L[q] = loaded(A, D, i, l, delta);
        step_lower(i, l, TS);
      }
    }
    __syncwarp();

    // ---- right-looking Cholesky, trailing updates spread over the team ----
    bool ok = true;
    for (int j = 0; j < D; ++j) {
      double djj = L[pidx(j, j)].x;
      if (!(djj > 0.0) || !isfinite(djj)) {
        ok = false;
        djj = 1.0;  // keep the control flow uniform; this system's weights become zero
      }
      const double inv = rsqrt(djj);
      const double ljj = djj * inv;
      for (int i = j + 1 + tl; i < D; i += TS) {
        const double2 v = L[pidx(i, j)];
        L[pidx(i, j)] = make_double2(v.x * inv, v.y * inv);
      }
      __syncwarp();
      const int m = D - j - 1;
      const int np = m * (m + 1) / 2;
      // entries (a, b) of the trailing triangle, two per iteration: they only
      // read column j, which this loop does not write, so both loads go first
      int a = 0, b = 0;
      step_lower(a, b, tl);
      for (int q = tl; q < np; q += 2 * TS) {
        int a2 = a, b2 = b;
        step_lower(a2, b2, TS);
        const bool two = q + TS < np;
        const int i = j + 1 + a, l = j + 1 + b;
        const int i2 = two ? j + 1 + a2 : i, l2 = two ? j + 1 + b2 : l;
        double2 acc = L[pidx(i, l)], acc2 = L[pidx(i2, l2)];
        const double2 lij = L[pidx(i, j)], llj = L[pidx(l, j)];
        const double2 lij2 = L[pidx(i2, j)], llj2 = L[pidx(l2, j)];
        // acc -= lij * conj(llj)
        acc.x = fma(-lij.x, llj.x, acc.x);
        acc2.x = fma(-lij2.x, llj2.x, acc2.x);
        acc.y = fma(-lij.y, llj.x, acc.y);
        acc2.y = fma(-lij2.y, llj2.x, acc2.y);
        acc.x = fma(-lij.y, llj.y, acc.x);
        acc2.x = fma(-lij2.y, llj2.y, acc2.x);
        acc.y = fma(lij.x, llj.y, acc.y);
        acc2.y = fma(lij2.x, llj2.y, acc2.y);
        L[pidx(i, l)] = acc;
        if (two) L[pidx(i2, l2)] = acc2;
        a = a2;
        b = b2;
        step_lower(a, b, TS);
      }
      __syncwarp();
      if (tl == 0) {
        L[pidx(j, j)] = make_double2(ljj, 0.0);
        invd[j] = inv;
      }
      __syncwarp();
    }

    // Weights of steering vector s from its solution u (stride 32): scale by
    // 1/sqrt(Re v_s^H u) and store as complex64.
    auto emit = [&](int s, const double2* u) {
      const double2* v = steer + (size_t)s * D;
      double q = 0.0;
      for (int i = 0; i < D; ++i) {
        const double2 vi = __ldg(v + i), ui = u[i * 32];
        q = fma(vi.x, ui.x, q);
        q = fma(vi.y, ui.y, q);
      }
      const bool good = ok && q > 0.0 && isfinite(q);
      const float sf = good ? (float)rsqrt(q) : 0.f;
      if (valid) {
        float2* w = wts + ((size_t)sys * S + s) * D;
        for (int i = 0; i < D; ++i) {
          const double2 ui = u[i * 32];
          if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2((float)ui.x * sf, (float)ui.y * sf) : make_float2(0.f, 0.f);
        }
      }
    };

    // ---- per-lane solves: one right-hand side per lane and pass ----
    // generic: the S steering vectors, each written as soon as it is solved;
    // SEP: the C <= TS basis vectors g (x) e_c, all in one pass
    const int nrhs = SEP ? C : S;
    for (int r0 = 0; r0 < nrhs; r0 += TS) {
      const int rhs = r0 + tl;
      if (rhs < nrhs) {
        const double2* v = steer + (size_t)rhs * D;
        auto rhs_at = [&](int i) -> double2 {
          if (SEP) {
            const int t = i / C;
            return (i - t * C == rhs) ? __ldg(sep_g + t) : make_double2(0.0, 0.0);
          }
          return __ldg(v + i);
        };
        for (int i = 0; i < D; ++i) W[i * 32] = rhs_at(i);
        chol_solve_inplace(L, invd, W, D);
        for (int i = 0; i < D; ++i) U[i * 32] = W[i * 32];
        for (int it = 0; it < refine_steps; ++it) {
          // W = b - Rl u  (Rl Hermitian: lower part direct, upper part mirrored)
          for (int i = 0; i < D; ++i) {
            double2 acc = rhs_at(i);
            for (int l = 0; l < i; ++l) cfms(acc, __ldg(A + (size_t)i * D + l), U[l * 32]);
            diag_fms(acc, __ldg(&A[(size_t)i * D + i].x) + delta, U[i * 32]);
            for (int l = i + 1; l < D; ++l) cfms_conj(acc, __ldg(A + (size_t)l * D + i), U[l * 32]);
            W[i * 32] = acc;
          }
          chol_solve_inplace(L, invd, W, D);
          for (int i = 0; i < D; ++i) {
            const double2 u = U[i * 32], c = W[i * 32];
            U[i * 32] = make_double2(u.x + c.x, u.y + c.y);
          }
        }
        if (!SEP) emit(rhs, U);
      }
    }

    // ---- SEP: combine the basis solutions (U_c = column of lane team*TS + c) ----
    if (SEP) {
      __syncwarp();
      float4* Wf = reinterpret_cast<float4*>(W);
      if (tl < C)
        for (int i = 0; i < D; ++i) Wf[i * 32] = to_ff4(U[i * 32]);
      __syncwarp();
      sep_emit(Wf - lane + team * TS, D, S, C, TS, tl, steer_ff, sep_a_ff, ok,
               valid ? wts + (size_t)sys * S * D : nullptr);
    }
    if (valid && !ok && tl == 0) atomicAdd(&status->n_failed, 1ULL);
    __syncwarp();  // the next batch reuses L, U, W
  }
}

template <bool SEP>
__global__ void __launch_bounds__(128)
solve_kernel(SolveParams p) {
  solve_kernel_body<SEP>(p, blockIdx.x, gridDim.x);
}

// the same solves as a persistent launch over the CPIs of a batch
template <bool SEP>
__global__ void __launch_bounds__(128)
solve_kernel_batched(BatchCtl ctl) {
  batched_loop<SolveParams>(ctl, [&](const SolveParams& p, int bx, int, int gx) {
    solve_kernel_body<SEP>(p, bx, gx);
  });
}

// ---------------------------------------------------------------------------
// Register-resident form for the common snapshot lengths (D = 8, 12, 16):
// the team mapping of solve_kernel, but with D a compile-time constant, every
// loop over it unrolled, and each lane's right-hand side, solution and
// residual held in registers.  The substitutions then read nothing but the
// factor from shared memory, and the compiler interleaves the rows (row i's
// partial sums start before x_{i-1} is final).  The factor is kept as
// Rl = Lu Dg Lu^H (unit lower Lu, real pivots Dg): no square roots, and the
// substitutions scale once, by Dg^{-1}, between the forward and the back
// pass.  Column j of the elimination divides by the pivot d_j and updates the
// trailing entries with l_ij conj(a_lj), a_lj the column before the division
// (= l_lj d_j), kept in a small per-team buffer.
template <int D, bool SEP>
__device__ __forceinline__ void solve_reg_kernel_body(const SolveParams& prm, long long bx, long long gx) {
  const double2* __restrict__ cov = prm.cov;
  float2* __restrict__ wts = prm.wts;
  const double2* __restrict__ steer = prm.steer;
  const double2* __restrict__ sep_g = prm.sep_g;
  const float4* __restrict__ steer_ff = prm.steer_ff;
  const float4* __restrict__ sep_a_ff = prm.sep_a_ff;
  const long long nsys = prm.nsys;
  const int S = prm.S, C = prm.C;
  const double load_factor = prm.load_factor;
  const int refine_steps = prm.refine_steps;
  DeviceStatus* __restrict__ status = prm.status;
  (void)steer; (void)sep_g; (void)steer_ff; (void)sep_a_ff;
  const int TS = prm.TS;
  constexpr int Dp = D * (D + 1) / 2;
  extern __shared__ double2 sm[];
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = 32 / TS, team = lane / TS, tl = lane - team * TS;
  // per warp: G factors [Dp], G pivot columns [D], (SEP) the [D][32] float4
  // exchange area for the combination; after all warps: G pivot reciprocals [D]
  const bool alias = G * Dp >= 32 * D;   // the exchange area fits over the factors
  const size_t warp_elems = (size_t)G * (Dp + D) + (SEP && !alias ? (size_t)D * 32 : 0);
  double2* wbase = sm + warp * warp_elems;
  double2* L = wbase + (size_t)team * Dp;
  double2* col = wbase + (size_t)G * Dp + (size_t)team * D;
  float4* Wf = reinterpret_cast<float4*>(alias ? wbase : wbase + (size_t)G * (Dp + D));
  double* rdp = reinterpret_cast<double*>(sm + nw * warp_elems) + ((size_t)warp * G + team) * D;

  for (long long base = ((long long)bx * nw + warp) * G; base < nsys;
       base += (long long)gx * nw * G) {
    const long long sys = base + team;
    const bool valid = sys < nsys;
    const double2* A = cov + (size_t)(valid ? sys : nsys - 1) * D * D;

    // ---- diagonal load and packed copy of Rl ----
    double tr = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) tr += __ldg(&A[j * D + j].x);
    const double delta = load_factor * tr * (1.0 / D);
    {
      int i = 0, l = 0;
      step_lower(i, l, tl);
      for (int q = tl; q < Dp; q += TS) {
        L[q] = loaded(A, D, i, l, delta);
        step_lower(i, l, TS);
      }
    }
    __syncwarp();

    // ---- Rl = Lu Dg Lu^H, trailing updates spread over the team ----
    bool ok = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double djj = L[pidx(j, j)].x;
      if (!(djj > 0.0) || !isfinite(djj)) {
        ok = false;
        djj = 1.0;  // keep the control flow uniform; this system's weights become zero
      }
      const double rd = 1.0 / djj;
      for (int i = j + 1 + tl; i < D; i += TS) {
        const double2 v = L[pidx(i, j)];
        col[i] = v;
        L[pidx(i, j)] = make_double2(v.x * rd, v.y * rd);
      }
      __syncwarp();
      const int m = D - 1 - j, np = m * (m + 1) / 2;
      int a = 0, b = 0;
      step_lower(a, b, tl);
      for (int q = tl; q < np; q += TS) {
        const int i = j + 1 + a, l = j + 1 + b;
        double2 acc = L[pidx(i, l)];
        const double2 lij = L[pidx(i, j)], alj = col[l];
        // acc -= lij * conj(alj)
        acc.x = fma(-lij.x, alj.x, acc.x);
        acc.x = fma(-lij.y, alj.y, acc.x);
        acc.y = fma(-lij.y, alj.x, acc.y);
        acc.y = fma(lij.x, alj.y, acc.y);
        L[pidx(i, l)] = acc;
        step_lower(a, b, TS);
      }
      if (tl == 0) rdp[j] = rd;
      __syncwarp();
    }

    // x <- Rl^{-1} x: Lu z = x, y = Dg^{-1} z, Lu^H x = y.  The warp
    // barriers between rows keep the compiler from hoisting every load of
    // the factor to the top (it would hold them all in registers and spill);
    // every lane of the warp runs them (see the pass loop below).
    auto ldl_solve = [&](double2 (&x)[D]) {
#pragma unroll
      for (int i = 1; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < i; ++l) cfms(x[i], L[pidx(i, l)], x[l]);
        __syncwarp();
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const double r = rdp[i];
        x[i].x *= r;
        x[i].y *= r;
      }
#pragma unroll
      for (int i = D - 2; i >= 0; --i) {
#pragma unroll
        for (int l = i + 1; l < D; ++l) cfms_conj(x[i], L[pidx(l, i)], x[l]);
        __syncwarp();
      }
    };

    // ---- per-lane solves: one right-hand side per lane and pass ----
    // Lanes past the last right-hand side solve a copy of the first one and
    // store nothing, so that the whole warp reaches the barriers together.
    const int nrhs = SEP ? C : S;
    for (int r0 = 0; r0 < nrhs; r0 += TS) {
      const bool live = r0 + tl < nrhs;
      const int rhs = live ? r0 + tl : 0;
      {
        auto rhs_at = [&](int i) -> double2 {
          if (SEP) {
            const int t = i / C;
            return (i - t * C == rhs) ? __ldg(sep_g + t) : make_double2(0.0, 0.0);
          }
          return __ldg(steer + (size_t)rhs * D + i);
        };
        double2 u[D], r[D];
#pragma unroll
        for (int i = 0; i < D; ++i) u[i] = rhs_at(i);
        ldl_solve(u);
        for (int it = 0; it < refine_steps; ++it) {
          // r = b - Rl u  (Rl Hermitian: lower part direct, upper part mirrored)
#pragma unroll
          for (int i = 0; i < D; ++i) {
            double2 acc = rhs_at(i);
#pragma unroll
            for (int l = 0; l < i; ++l) cfms(acc, __ldg(A + i * D + l), u[l]);
            diag_fms(acc, __ldg(&A[i * D + i].x) + delta, u[i]);
#pragma unroll
            for (int l = i + 1; l < D; ++l) cfms_conj(acc, __ldg(A + l * D + i), u[l]);
            r[i] = acc;
            __syncwarp();
          }
          ldl_solve(r);
#pragma unroll
          for (int i = 0; i < D; ++i) {
            u[i].x += r[i].x;
            u[i].y += r[i].y;
          }
        }
        if (SEP) {
          __syncwarp();   // every lane is done with the factors the area may overlay
          if (live)
#pragma unroll
            for (int i = 0; i < D; ++i) Wf[i * 32 + lane] = to_ff4(u[i]);
        } else {
          const double2* v = steer + (size_t)rhs * D;
          double q = 0.0;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const double2 vi = __ldg(v + i);
            q = fma(vi.x, u[i].x, q);
            q = fma(vi.y, u[i].y, q);
          }
          const bool good = ok && q > 0.0 && isfinite(q);
          const float sf = good ? (float)rsqrt(q) : 0.f;
          if (valid && live) {
            float2* w = wts + ((size_t)sys * S + rhs) * D;
#pragma unroll
            for (int i = 0; i < D; ++i)
              if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2((float)u[i].x * sf, (float)u[i].y * sf) : make_float2(0.f, 0.f);
          }
        }
      }
    }
    if (SEP) {
      __syncwarp();
      sep_emit(Wf + team * TS, D, S, C, TS, tl, steer_ff, sep_a_ff, ok,
               valid ? wts + (size_t)sys * S * D : nullptr);
    }
    if (valid && !ok && tl == 0) atomicAdd(&status->n_failed, 1ULL);
    __syncwarp();  // the next batch reuses L, col, Wf
  }
}

template <int D, bool SEP>
__global__ void __launch_bounds__(128, 4)
solve_reg_kernel(SolveParams p) {
  solve_reg_kernel_body<D, SEP>(p, blockIdx.x, gridDim.x);
}

// the same solves as a persistent launch over the CPIs of a batch
template <int D, bool SEP>
__global__ void __launch_bounds__(128, 4)
solve_reg_kernel_batched(BatchCtl ctl) {
  batched_loop<SolveParams>(ctl, [&](const SolveParams& p, int bx, int, int gx) {
    solve_reg_kernel_body<D, SEP>(p, bx, gx);
  });
}

// ---------------------------------------------------------------------------
// Mixed-precision iterative refinement (STAP_SOLVE_MIXED_IR) for D = 8, 12,
// 16, with the team mapping and register-resident vectors of
// solve_reg_kernel.  The loaded matrix Rl is kept in shared memory as
// double-floats (hi + lo, about 2^-48 relative) and its FP32 part is factored
// as Lu Dg Lu^H in FP32.  Each right-hand side b is solved in FP32; then
// every refinement step forms the residual r = b - Rl u in double-float on
// the FP32 pipe, solves Rl c = r in FP32 and adds c to the double-float
// solution u (the classical three-precision scheme: factorisation 2^-24,
// working and residual precision 2^-48).  Each step shrinks the error by
// about kappa(Rl) 2^-24; with the clutter conditioning kappa ~ 1e3 D, two
// steps reach the FP32 rounding of the stored weights.  The FP64 pipe only
// adds the diagonal load and splits the input.
__host__ __device__ constexpr size_t mir_warp_bytes(int D, int G, bool sep) {
  // G double-float matrices [Dp] (the SEP exchange area [D][32] float4
  // overlays them when they are large enough, else follows), G FP32 factors
  // [Dp], the per-lane residual columns [D][32] float2, G pivot columns [D]
  // float2, G pivot reciprocals [D] float; per-team strides odd_up(Dp) and
  // odd_up(D)
  return ((size_t)G * odd_up(D * (D + 1) / 2) +
          (sep && G * odd_up(D * (D + 1) / 2) < 32 * D ? (size_t)D * 32 : 0)) * 16 +
         ((size_t)G * odd_up(D * (D + 1) / 2) * 8 + 15) / 16 * 16 + (size_t)D * 32 * 8 +
         ((size_t)G * odd_up(D) * 8 + 15) / 16 * 16 + ((size_t)G * odd_up(D) * 4 + 15) / 16 * 16;
}

// A compensated sum of double-float products (Dot2 of Ogita, Rump and Oishi,
// extended to double-float factors): s collects the rounded products with
// TwoSum, e every rounding error and the cross terms; the value is s + e.
struct Dot2 {
  float s, e;
};

// acc += (ah + al) * (bh + bl), dropping al * bl (below 2^-48 of the product)
__device__ __forceinline__ void dot2_add(Dot2& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float t = __fadd_rn(acc.s, p);
  const float z = __fsub_rn(t, acc.s);
  const float te = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, z)), __fsub_rn(p, z));
  acc.s = t;
  acc.e = __fadd_rn(acc.e, __fadd_rn(te, pe));
}

// accr + i acci -= a * u   (a = (re_hi, re_lo, im_hi, im_lo), u = ur + i ui)
__device__ __forceinline__ void dot2_cfms(Dot2& accr, Dot2& acci, float4 a, ff::F2 ur, ff::F2 ui) {
  dot2_add(accr, -a.x, -a.y, ur.hi, ur.lo);
  dot2_add(accr, a.z, a.w, ui.hi, ui.lo);
  dot2_add(acci, -a.x, -a.y, ui.hi, ui.lo);
  dot2_add(acci, -a.z, -a.w, ur.hi, ur.lo);
}

template <int D, bool SEP>
__global__ void __launch_bounds__(128, 4)
solve_mir_kernel(const double2* __restrict__ cov, float2* __restrict__ wts,
                 const float4* __restrict__ steer_ff, const float4* __restrict__ g_ff,
                 const float4* __restrict__ sep_a_ff, long long nsys, int S, int C, int TS,
                 double load_factor, int refine_steps, DeviceStatus* __restrict__ status) {
  constexpr int Dp = D * (D + 1) / 2;
  extern __shared__ float4 smf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int G = 32 / TS, team = lane / TS, tl = lane - team * TS;
  constexpr int LS = odd_up(Dp), CS = odd_up(D);   // per-team strides
  const bool alias = G * LS >= 32 * D;
  char* wb = reinterpret_cast<char*>(smf) + warp * mir_warp_bytes(D, G, SEP);
  float4* Ad = reinterpret_cast<float4*>(wb) + (size_t)team * LS;
  float4* Wf = reinterpret_cast<float4*>(wb) + (alias ? 0 : (size_t)G * LS);
  char* fb = wb + ((size_t)G * LS + (SEP && !alias ? (size_t)D * 32 : 0)) * 16;
  float2* Lf = reinterpret_cast<float2*>(fb) + (size_t)team * LS;
  char* rb = fb + ((size_t)G * LS * 8 + 15) / 16 * 16;
  float2* Rs = reinterpret_cast<float2*>(rb) + lane;     // [D][32]
  char* pb = rb + (size_t)D * 32 * 8;
  float2* colf = reinterpret_cast<float2*>(pb) + (size_t)team * CS;
  float* rdf = reinterpret_cast<float*>(pb + ((size_t)G * CS * 8 + 15) / 16 * 16) + (size_t)team * CS;

  for (long long base = ((long long)blockIdx.x * nw + warp) * G; base < nsys;
       base += (long long)gridDim.x * nw * G) {
    const long long sys = base + team;
    const bool valid = sys < nsys;
    const double2* A = cov + (size_t)(valid ? sys : nsys - 1) * D * D;

    // ---- Rl as double-floats and its FP32 part ----
    double tr = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) tr += __ldg(&A[j * D + j].x);
    const double delta = load_factor * tr * (1.0 / D);
    {
      int i = 0, l = 0;
      step_lower(i, l, tl);
      for (int q = tl; q < Dp; q += TS) {
        const float4 f = to_ff4_cvt(loaded(A, D, i, l, delta));
        Ad[q] = f;
        Lf[q] = make_float2(f.x, f.z);
        step_lower(i, l, TS);
      }
    }
    __syncwarp();

    // ---- FP32 Lu Dg Lu^H ----
    bool ok = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float djj = Lf[pidx(j, j)].x;
      if (!(djj > 0.f) || !isfinite(djj)) {
        ok = false;
        djj = 1.f;
      }
      const float rd = 1.0f / djj;
      for (int i = j + 1 + tl; i < D; i += TS) {
        const float2 v = Lf[pidx(i, j)];
        colf[i] = v;
        Lf[pidx(i, j)] = make_float2(v.x * rd, v.y * rd);
      }
      __syncwarp();
      const int m = D - 1 - j, np = m * (m + 1) / 2;
      int a = 0, b = 0;
      step_lower(a, b, tl);
      for (int q = tl; q < np; q += TS) {
        const int i = j + 1 + a, l = j + 1 + b;
        float2 acc = Lf[pidx(i, l)];
        const float2 lij = Lf[pidx(i, j)], alj = colf[l];
        acc.x = fmaf(-lij.x, alj.x, acc.x);
        acc.x = fmaf(-lij.y, alj.y, acc.x);
        acc.y = fmaf(-lij.y, alj.x, acc.y);
        acc.y = fmaf(lij.x, alj.y, acc.y);
        Lf[pidx(i, l)] = acc;
        step_lower(a, b, TS);
      }
      if (tl == 0) rdf[j] = rd;
      __syncwarp();
    }

    // x <- Rl^{-1} x in FP32 (warp barriers between rows, as in solve_reg_kernel)
    auto f32_solve = [&](float2 (&x)[D]) {
#pragma unroll
      for (int i = 1; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < i; ++l) {
          const float2 a = Lf[pidx(i, l)];
          x[i].x = fmaf(-a.x, x[l].x, x[i].x);
          x[i].x = fmaf(a.y, x[l].y, x[i].x);
          x[i].y = fmaf(-a.x, x[l].y, x[i].y);
          x[i].y = fmaf(-a.y, x[l].x, x[i].y);
        }
        __syncwarp();
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const float r = rdf[i];
        x[i].x *= r;
        x[i].y *= r;
      }
#pragma unroll
      for (int i = D - 2; i >= 0; --i) {
#pragma unroll
        for (int l = i + 1; l < D; ++l) {
          const float2 a = Lf[pidx(l, i)];
          x[i].x = fmaf(-a.x, x[l].x, x[i].x);
          x[i].x = fmaf(-a.y, x[l].y, x[i].x);
          x[i].y = fmaf(-a.x, x[l].y, x[i].y);
          x[i].y = fmaf(a.y, x[l].x, x[i].y);
        }
        __syncwarp();
      }
    };

    // ---- per-lane right-hand sides (idle lanes repeat the first one) ----
    const int nrhs = SEP ? C : S;
    for (int r0 = 0; r0 < nrhs; r0 += TS) {
      const bool live = r0 + tl < nrhs;
      const int rhs = live ? r0 + tl : 0;
      auto rhs_ff = [&](int i) -> float4 {
        if (SEP) {
          const int t = i / C;
          return (i - t * C == rhs) ? __ldg(g_ff + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return __ldg(steer_ff + (size_t)rhs * D + i);
      };
      float2 x[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const float4 b = rhs_ff(i);
        x[i] = make_float2(b.x, b.z);
      }
      f32_solve(x);
      ff::F2 ur[D], ui[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        ur[i] = ff::F2{x[i].x, 0.f};
        ui[i] = ff::F2{x[i].y, 0.f};
      }
      for (int it = 0; it < refine_steps; ++it) {
        // x = fl32(b - Rl u), the residual formed in double-float.  The row
        // loop is not unrolled (fully unrolled it is too large, and the
        // solution would leave the registers); row i goes to this lane's
        // column of Rs.  Above the diagonal Rl[i][l] = conj(Rl[l][i]).
        // Two compensated sums per component (even and odd l) keep two
        // independent dependency chains in flight.
        for (int i = 0; i < D; ++i) {
          const float4 b = rhs_ff(i);
          Dot2 rr{b.x, b.y}, ri{b.z, b.w}, rr2{0.f, 0.f}, ri2{0.f, 0.f};
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const bool low = l <= i;
            float4 a = Ad[low ? pidx(i, l) : pidx(l, i)];
            if (!low) {
              a.z = -a.z;
              a.w = -a.w;
            }
            if (l & 1) dot2_cfms(rr2, ri2, a, ur[l], ui[l]);
            else dot2_cfms(rr, ri, a, ur[l], ui[l]);
          }
          const float xr = __fadd_rn(__fadd_rn(rr.s, rr2.s), __fadd_rn(rr.e, rr2.e));
          const float xi = __fadd_rn(__fadd_rn(ri.s, ri2.s), __fadd_rn(ri.e, ri2.e));
          Rs[i * 32] = make_float2(xr, xi);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = Rs[i * 32];
        f32_solve(x);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          ur[i] = ff::add(ur[i], x[i].x);
          ui[i] = ff::add(ui[i], x[i].y);
        }
      }
      if (SEP) {
        __syncwarp();   // every lane is done with Ad, which the exchange area may overlay
        if (live)
#pragma unroll
          for (int i = 0; i < D; ++i) Wf[i * 32 + lane] = make_float4(ur[i].hi, ur[i].lo, ui[i].hi, ui[i].lo);
      } else {
        ff::F2 q{0.f, 0.f};                       // Re v^H u
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const float4 v = __ldg(steer_ff + (size_t)rhs * D + i);
          q = ff::fma(ff::fma(q, ff::F2{v.x, v.y}, ur[i]), ff::F2{v.z, v.w}, ui[i]);
        }
        const double qd = ff::to_double(q);
        const bool good = ok && qd > 0.0 && isfinite(qd);
        const float sf = good ? (float)rsqrt(qd) : 0.f;
        if (valid && live) {
          float2* w = wts + ((size_t)sys * S + rhs) * D;
#pragma unroll
          for (int i = 0; i < D; ++i)
            if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2(__fadd_rn(ur[i].hi, ur[i].lo) * sf, __fadd_rn(ui[i].hi, ui[i].lo) * sf)
                        : make_float2(0.f, 0.f);
        }
      }
    }
    if (SEP) {
      __syncwarp();
      sep_emit(Wf + team * TS, D, S, C, TS, tl, steer_ff, sep_a_ff, ok,
               valid ? wts + (size_t)sys * S * D : nullptr);
    }
    if (valid && !ok && tl == 0) atomicAdd(&status->n_failed, 1ULL);
    __syncwarp();  // the next batch reuses Ad, Lf, colf, Wf
  }
}

// ---------------------------------------------------------------------------
// Larger systems (32 < D <= 128).  The per-lane layout above needs two D-long
// FP64 vectors per lane, which stops fitting next to the factor, so here one
// CTA of 4 (or 8) warps owns one system at a time and the lanes own ROWS:
//  * The factor lives in shared memory as Rl = Lu Dg Lu^H (unit lower Lu,
//    column-major packed, and the pivot reciprocals 1/d_j).  The elimination
//    is right-looking with the trailing update of each column spread over
//    all threads; it divides column j by d_j and updates with l_ij conj(a_lj),
//    a_lj the column before the division.  The thread that updates the next
//    pivot also forms its reciprocal, so no square root and one division per
//    column.
//  * A group of LR lanes (LR = 32, or 16 for D <= 64 so that a warp carries
//    two right-hand sides) solves one right-hand side at a time; lane l of
//    the group keeps rows l, l + LR, l + 2 LR, l + 3 LR of its vectors in
//    registers.  Substitution goes column by column: the owner of row j
//    holds x_j, a shuffle broadcasts it, and the group updates its rows below
//    (above, for Lu^H); with a unit diagonal there is no per-column scaling,
//    only one Dg^{-1} scaling of every row between the two passes.
//  * The residual b - Rl u reads Rl from the input through L1: for each
//    column index l every lane takes A[i][l] (i >= l) or conj(A[l][i]) (i < l)
//    by a select, so all lanes run every DFMA.
//  * Separable steering: the C basis solutions are kept in shared memory as
//    double-floats and combined per steering vector, with the normalisation,
//    on the FP32 pipe (as in the small-system kernels).

__device__ __forceinline__ int colstart(int l, int D) { return l * D - l * (l - 1) / 2; }

// In-place forward (Lu z = x) or back (Lu^H z = x) substitution with the unit
// lower factor, of one vector held as rows li + LR q by the LR lanes of group
// `grp` (li = lane % LR).  The columns go in blocks of LR: block qb's columns
// live in register x[qb] of the group's lanes (a shuffle broadcasts x_j), and
// only the row blocks the block's columns update are visited -- q >= qb
// forward, q <= qb back -- with the block indices compile-time constants, so
// no FP64 instruction is issued for a row block with nothing to do (a warp
// FP64 instruction costs the same with no lane active).
template <int LR, int RPL, bool BACK>
__device__ __forceinline__ void big_subst(double2 (&x)[RPL], const double2* __restrict__ Lc,
                                          int D, int li, int grp) {
#pragma unroll
  for (int bb = 0; bb < RPL; ++bb) {
    const int qb = BACK ? RPL - 1 - bb : bb;
    if (LR * qb >= D) continue;                           // warp-uniform
    const int jn = min(LR, D - LR * qb);
    for (int jj = 0; jj < jn; ++jj) {
      const int jo = BACK ? jn - 1 - jj : jj;
      const int j = LR * qb + jo;
      double2 yj;
      yj.x = __shfl_sync(0xffffffffu, x[qb].x, grp * LR + jo);
      yj.y = __shfl_sync(0xffffffffu, x[qb].y, grp * LR + jo);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        if (BACK ? (q > qb) : (q < qb)) continue;         // compile-time
        if (LR * q >= D) continue;                        // warp-uniform
        const int i = li + LR * q;
        const bool act = BACK ? (i < j) : (i > j && i < D);
        if (act) {
          if (BACK) {  // x_i -= conj(Lu[j][i]) x_j
            const double2 l = Lc[colstart(i, D) + j - i];
            x[q].x = fma(-l.x, yj.x, x[q].x);
            x[q].x = fma(-l.y, yj.y, x[q].x);
            x[q].y = fma(-l.x, yj.y, x[q].y);
            x[q].y = fma(l.y, yj.x, x[q].y);
          } else {     // x_i -= Lu[i][j] x_j
            const double2 l = Lc[colstart(j, D) + i - j];
            x[q].x = fma(-l.x, yj.x, x[q].x);
            x[q].x = fma(l.y, yj.y, x[q].x);
            x[q].y = fma(-l.x, yj.y, x[q].y);
            x[q].y = fma(-l.y, yj.x, x[q].y);
          }
        }
      }
    }
  }
}

// x <- Rl^{-1} x with Rl = Lu Dg Lu^H (rd: the pivot reciprocals).
template <int LR, int RPL>
__device__ __forceinline__ void big_solve(double2 (&x)[RPL], const double2* __restrict__ Lc,
                                          const double* __restrict__ rd, int D, int li, int grp) {
  big_subst<LR, RPL, false>(x, Lc, D, li, grp);
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    if (LR * q < D) {
      const int i = li + LR * q;
      const double r = rd[i < D ? i : D - 1];
      x[q].x *= r;
      x[q].y *= r;
    }
  }
  big_subst<LR, RPL, true>(x, Lc, D, li, grp);
}

template <int LR>
__device__ __forceinline__ double group_sum(double v) {
  for (int o = LR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place FP32 forward (Lu z = x) or back (Lu^H z = x) substitution, as big_subst.
template <int LR, int RPL, bool BACK>
__device__ __forceinline__ void big_subst_f32(float2 (&x)[RPL], const float2* __restrict__ Lc,
                                              int D, int li, int grp) {
#pragma unroll
  for (int bb = 0; bb < RPL; ++bb) {
    const int qb = BACK ? RPL - 1 - bb : bb;
    if (LR * qb >= D) continue;
    const int jn = min(LR, D - LR * qb);
    for (int jj = 0; jj < jn; ++jj) {
      const int jo = BACK ? jn - 1 - jj : jj;
      const int j = LR * qb + jo;
      float2 yj;
      yj.x = __shfl_sync(0xffffffffu, x[qb].x, grp * LR + jo);
      yj.y = __shfl_sync(0xffffffffu, x[qb].y, grp * LR + jo);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        if (BACK ? (q > qb) : (q < qb)) continue;
        if (LR * q >= D) continue;
        const int i = li + LR * q;
        const bool act = BACK ? (i < j) : (i > j && i < D);
        if (act) {
          if (BACK) {
            const float2 l = Lc[colstart(i, D) + j - i];
            x[q].x = fmaf(-l.x, yj.x, x[q].x);
            x[q].x = fmaf(-l.y, yj.y, x[q].x);
            x[q].y = fmaf(-l.x, yj.y, x[q].y);
            x[q].y = fmaf(l.y, yj.x, x[q].y);
          } else {
            const float2 l = Lc[colstart(j, D) + i - j];
            x[q].x = fmaf(-l.x, yj.x, x[q].x);
            x[q].x = fmaf(l.y, yj.y, x[q].x);
            x[q].y = fmaf(-l.x, yj.y, x[q].y);
            x[q].y = fmaf(-l.y, yj.x, x[q].y);
          }
        }
      }
    }
  }
}

template <int LR, int RPL>
__device__ __forceinline__ void big_solve_f32(float2 (&x)[RPL], const float2* __restrict__ Lc,
                                              const float* __restrict__ rd, int D, int li, int grp) {
  big_subst_f32<LR, RPL, false>(x, Lc, D, li, grp);
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    if (LR * q < D) {
      const int i = li + LR * q;
      const float r = rd[i < D ? i : D - 1];
      x[q].x *= r;
      x[q].y *= r;
    }
  }
  big_subst_f32<LR, RPL, true>(x, Lc, D, li, grp);
}

// F32F: the refinement option's form for D > 64 (where solve_big_mir_kernel's
// layout, with the broadcast area and the basis solutions beside the
// double-float matrix, does not fit in shared memory): the factor and the
// substitutions in FP32, the solution in FP64, each refinement step's
// residual in double-float from a double-float copy of Rl kept in shared
// memory where the FP64 kernel keeps the basis solutions, its FP32
// correction added in FP64.  With separable steering the basis solutions are
// parked in the system's own weight rows (which hold S D >= 2 C D floats)
// until every right-hand side is done, then copied over the matrix copy for
// the combination.  256-thread CTAs hold a D > 64 system's factor (one CTA
// per SM), so they may use the whole register file; 128-thread CTAs run
// three per SM.
template <bool SEP, int LR, int NT, int RPL, bool F32F>
__device__ __forceinline__ void solve_big_kernel_body(const SolveParams& prm, long long bx, long long gx) {
  const double2* __restrict__ cov = prm.cov;
  float2* __restrict__ wts = prm.wts;
  const double2* __restrict__ steer = prm.steer;
  const double2* __restrict__ sep_g = prm.sep_g;
  const float4* __restrict__ steer_ff = prm.steer_ff;
  const float4* __restrict__ sep_a_ff = prm.sep_a_ff;
  const long long nsys = prm.nsys;
  const int S = prm.S, C = prm.C;
  const double load_factor = prm.load_factor;
  const int refine_steps = prm.refine_steps;
  DeviceStatus* __restrict__ status = prm.status;
  (void)steer; (void)sep_g; (void)steer_ff; (void)sep_a_ff;
  const int D = prm.D;
  using LT = typename std::conditional<F32F, float2, double2>::type;   // factor entries
  using RT = typename std::conditional<F32F, float, double>::type;     // pivots
  extern __shared__ double2 sm[];
  constexpr int NW = NT / 32;
  constexpr int NG = NT / LR;                      // right-hand sides in flight per CTA
  const int Dp = D * (D + 1) / 2;
  // Lu [Dp] (column-major packed) and the two pivot columns before division [2][D];
  // from the next 16-byte boundary the SEP basis solutions [C][D]
  // (double-float) -- F32F: the loaded Rl [Dp] (double-float, column-major
  // packed), which the basis solutions overwrite for the combination -- the
  // pivot reciprocals [D] and the pivot flag
  LT* Lc = reinterpret_cast<LT*>(sm);
  LT* colb = Lc + Dp;                              // columns j and j+1 before division
  LT* colb2 = colb + D;
  float4* Ubf = reinterpret_cast<float4*>(sm) + ((size_t)(Dp + 2 * D) * sizeof(LT) + 15) / 16;
  float4* Adf = Ubf;
  RT* rd = reinterpret_cast<RT*>(Ubf + (F32F ? (size_t)Dp : (SEP ? (size_t)C * D : 0)));
  int* okf = reinterpret_cast<int*>(rd + D);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int li = lane % LR, grp = lane / LR;         // lane in group, group in warp
  const int g = warp * (32 / LR) + grp;              // group in CTA
  const double invD = 1.0 / (double)D;

  // pivot d -> reciprocal, recording a pivot that is not positive and finite
  auto pivot = [&](RT d) -> RT {
    if (!(d > RT(0)) || !isfinite(d)) {
      *okf = 0;
      return RT(1);  // keep going; this system's weights become zero
    }
    if constexpr (F32F) return RT(1) / d;
    else return recip_newton(d);
  };

  for (long long sys = bx; sys < nsys; sys += gx) {
    const double2* A = cov + (size_t)sys * D * D;
    double tr = 0.0;
    for (int j = 0; j < D; ++j) tr += __ldg(&A[(size_t)j * D + j].x);
    const double delta = load_factor * tr * invD;
    for (int i = warp; i < D; i += NW)                 // rows of A, coalesced
      for (int l = lane; l <= i; l += 32) {
        const double2 a = loaded(A, D, i, l, delta);
        Lc[colstart(l, D) + i - l] = LT{(RT)a.x, (RT)a.y};
        if constexpr (F32F) Adf[colstart(l, D) + i - l] = to_ff4_cvt(a);
      }
    if (tid == 0) *okf = 1;
    __syncthreads();

    // Right-looking Lu Dg Lu^H, two columns per round (two barriers per two
    // columns instead of four).  Phase 1: the thread of row i > j scales
    // column j (l_ij = a_ij / d_j), brings column j+1 up to date with it and
    // scales that too; every thread forms d_j, d_{j+1} and their reciprocals
    // itself from the same shared values and with the same operations (so
    // with the same bits), which keeps the reciprocals off the path between
    // the barriers.  l_{j+1,j} is read by every thread in phase 1, so its
    // owner stores it only in phase 2.  Phase 2: the rank-2 update of the
    // trailing triangle (columns >= j+2).
    for (int j = 0; j < D; j += 2) {
      const int cj = colstart(j, D);
      const int j1 = j + 1;
      const bool pair = j1 < D;
      const int c1 = pair ? colstart(j1, D) : cj;
      // only threads with a row in phase 1 (and thread 0, which stores the
      // reciprocals) need them: FP64 work costs per warp instruction
      const bool rows = j1 + tid < D || tid == 0;
      const RT rj = rows ? pivot(Lc[cj].x) : RT(1);
      LT a1j{RT(0), RT(0)};
      RT r1 = RT(1);
      if (pair && rows) {
        a1j = Lc[cj + 1];                                    // a_{j+1,j}
        const LT l1j{a1j.x * rj, a1j.y * rj};
        RT d1 = Lc[c1].x;
        d1 = fma(-l1j.x, a1j.x, d1);
        d1 = fma(-l1j.y, a1j.y, d1);
        r1 = pivot(d1);
      }
      LT l1j_own{RT(0), RT(0)};
      bool own1 = false;
      for (int i = j1 + tid; i < D; i += NT) {
        const LT v = Lc[cj + i - j];
        colb[i] = v;
        const LT lij{v.x * rj, v.y * rj};
        if (i == j1) {
          l1j_own = lij;
          own1 = true;
        } else {
          Lc[cj + i - j] = lij;
          // a_{i,j+1} -= l_ij conj(a_{j+1,j}); then l_{i,j+1} = a_{i,j+1} / d_{j+1}
          LT w = Lc[c1 + i - j1];
          w.x = fma(-lij.x, a1j.x, w.x);
          w.y = fma(-lij.y, a1j.x, w.y);
          w.x = fma(-lij.y, a1j.y, w.x);
          w.y = fma(lij.x, a1j.y, w.y);
          colb2[i] = w;
          Lc[c1 + i - j1] = LT{w.x * r1, w.y * r1};
        }
      }
      if (tid == 0) {
        rd[j] = rj;
        if (pair) rd[j1] = r1;
      }
      __syncthreads();
      if (own1) Lc[cj + 1] = l1j_own;
      // rank-2 update, pairs (i, l) with j+1 < l <= i, column-major order:
      // column a of the trailing triangle holds m - a entries; a thread steps
      // through its entries (a, off) NT at a time, two per iteration (they
      // read only columns j, j+1, colb and colb2, which this loop does not
      // write)
      const int m = D - j - 2;
      if (m > 0) {
        const int np = m * (m + 1) / 2;
        int a = 0, off = tid;
        while (a < m && off >= m - a) off -= m - a++;
        for (int q = tid; q < np; q += 2 * NT) {
          int a2 = a, off2 = off + NT;
          while (a2 < m && off2 >= m - a2) off2 -= m - a2++;
          const bool two = q + NT < np;
          const int l = j + 2 + a, i = l + off;
          const int l2 = two ? j + 2 + a2 : l, i2 = two ? l2 + off2 : i;
          const LT lij = Lc[cj + i - j], alj = colb[l], mij = Lc[c1 + i - j1], blj = colb2[l];
          const LT lij2 = Lc[cj + i2 - j], alj2 = colb[l2], mij2 = Lc[c1 + i2 - j1], blj2 = colb2[l2];
          LT acc = Lc[colstart(l, D) + i - l], acc2 = Lc[colstart(l2, D) + i2 - l2];
          // acc -= lij conj(alj) + mij conj(blj)
          acc.x = fma(-lij.x, alj.x, acc.x);
          acc2.x = fma(-lij2.x, alj2.x, acc2.x);
          acc.y = fma(-lij.y, alj.x, acc.y);
          acc2.y = fma(-lij2.y, alj2.x, acc2.y);
          acc.x = fma(-lij.y, alj.y, acc.x);
          acc2.x = fma(-lij2.y, alj2.y, acc2.x);
          acc.y = fma(lij.x, alj.y, acc.y);
          acc2.y = fma(lij2.x, alj2.y, acc2.y);
          acc.x = fma(-mij.x, blj.x, acc.x);
          acc2.x = fma(-mij2.x, blj2.x, acc2.x);
          acc.y = fma(-mij.y, blj.x, acc.y);
          acc2.y = fma(-mij2.y, blj2.x, acc2.y);
          acc.x = fma(-mij.y, blj.y, acc.x);
          acc2.x = fma(-mij2.y, blj2.y, acc2.x);
          acc.y = fma(mij.x, blj.y, acc.y);
          acc2.y = fma(mij2.x, blj2.y, acc2.y);
          Lc[colstart(l, D) + i - l] = acc;
          if (two) Lc[colstart(l2, D) + i2 - l2] = acc2;
          a = a2;
          off = off2 + NT;
          while (a < m && off >= m - a) off -= m - a++;
        }
      }
      __syncthreads();
    }
    const bool ok = *okf != 0;

    // weights of steering vector s from u (rows li + LR q): group-wide, and
    // called by every group (the sum shuffles across the whole warp); only a
    // live group stores
    auto emit = [&](int s, const double2 (&u)[RPL], bool live) {
      const double2* v = steer + (size_t)s * D;
      double qp = 0.0;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = li + LR * q;
        if (i < D) {
          const double2 vi = __ldg(v + i);
          qp = fma(vi.x, u[q].x, qp);
          qp = fma(vi.y, u[q].y, qp);
        }
      }
      const double qs = group_sum<LR>(qp);
      const bool good = ok && qs > 0.0 && isfinite(qs);
      const double scale = good ? rsqrt(qs) : 0.0;
      if (!live) return;
      float2* w = wts + ((size_t)sys * S + s) * D;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = li + LR * q;
        if (i < D)
          if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2((float)(u[q].x * scale), (float)(u[q].y * scale))
                      : make_float2(0.f, 0.f);
      }
    };

    // every group runs the same number of passes (shuffles need the whole warp)
    const int nrhs = SEP ? C : S;
    for (int r0 = 0; r0 < nrhs; r0 += NG) {
      const int rhs = r0 + g;
      const bool live = rhs < nrhs;
      const int rsafe = live ? rhs : 0;
      double2 b[RPL], u[RPL], r[RPL];
      float2 xf[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = li + LR * q;
        double2 v = make_double2(0.0, 0.0);
        if (i < D) {
          if (SEP) {
            const int t = i / C;
            if (i - t * C == rsafe) v = __ldg(sep_g + t);
          } else {
            v = __ldg(steer + (size_t)rsafe * D + i);
          }
        }
        b[q] = v;
        u[q] = v;
      }
      if constexpr (F32F) {   // FP32 solve of the rounded right-hand side
#pragma unroll
        for (int q = 0; q < RPL; ++q) xf[q] = make_float2((float)u[q].x, (float)u[q].y);
        big_solve_f32<LR, RPL>(xf, Lc, rd, D, li, grp);
#pragma unroll
        for (int q = 0; q < RPL; ++q) u[q] = make_double2(xf[q].x, xf[q].y);
      } else {
        big_solve<LR, RPL>(u, Lc, rd, D, li, grp);
      }
      for (int it = 0; it < refine_steps; ++it) {
        if constexpr (F32F) {
          // r = b - Rl u in double-float arithmetic (about 2^-48) on the FP32
          // pipe, from the double-float Rl in shared memory (the lower
          // triangle, the conjugate above it by a sign flip, the load
          // included); u split once per step and broadcast by shuffles
          ff::F2 rre[RPL], rim[RPL];
          float4 uf[RPL];
          int csi[RPL];                                   // start of column i (the upper part's reads)
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            uf[q] = to_ff4_cvt(u[q]);
            rre[q] = ff::from_double_cvt(b[q].x);
            rim[q] = ff::from_double_cvt(b[q].y);
            const int i = li + LR * q;
            csi[q] = colstart(i < D ? i : D - 1, D);
          }
#pragma unroll
          for (int ql = 0; ql < RPL; ++ql) {
            if (LR * ql >= D) break;
#pragma unroll 2
            for (int lo = 0; lo < LR; ++lo) {
            const int l = LR * ql + lo;
            if (l >= D) break;
            const int src = grp * LR + lo;
            const ff::F2 ur{__shfl_sync(0xffffffffu, uf[ql].x, src), __shfl_sync(0xffffffffu, uf[ql].y, src)};
            const ff::F2 ui{__shfl_sync(0xffffffffu, uf[ql].z, src), __shfl_sync(0xffffffffu, uf[ql].w, src)};
            const int cl = colstart(l, D);
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
              if (LR * q < D) {
                const int i = li + LR * q;
                const int ic = i < D ? i : D - 1;
                // row block q against column block ql: below it every entry is
                // in the lower triangle, above it in the upper (compile-time);
                // only the diagonal block decides per lane
                const bool low = q > ql ? true : (q < ql ? false : ic >= l);
                const int ao = low ? cl + ic - l : csi[q] + l - ic;
                const float4 e = in_bounds(ao, Dp, kSiteSolveIn) ? Adf[ao] : make_float4(0.f, 0.f, 0.f, 0.f);
                const ff::F2 nar{-e.x, -e.y};
                const ff::F2 ai = low ? ff::F2{e.z, e.w} : ff::F2{-e.z, -e.w};   // conj above the diagonal
                const ff::F2 nai{-ai.hi, -ai.lo};
                // r -= R[i][l] u_l:  re -= ar ur - ai ui,  im -= ar ui + ai ur
                rre[q] = ff::fma(ff::fma(rre[q], nar, ur), ai, ui);
                rim[q] = ff::fma(ff::fma(rim[q], nar, ui), nai, ur);
              }
            }
            }
          }
#pragma unroll
          for (int q = 0; q < RPL; ++q)
            xf[q] = make_float2(__fadd_rn(rre[q].hi, rre[q].lo), __fadd_rn(rim[q].hi, rim[q].lo));
        } else {
        // r = b - R u - delta u  (R Hermitian: A[i][l] for i >= l, conj(A[l][i])
        // above, real diagonal; the load is applied after the sweep)
#pragma unroll
        for (int q = 0; q < RPL; ++q) r[q] = b[q];
        // u_l lives in register ql = l / LR of the group's lane l % LR: a
        // shuffle broadcasts it (the loops' bounds are warp-uniform)
#pragma unroll
        for (int ql = 0; ql < RPL; ++ql) {
          if (LR * ql >= D) break;
#pragma unroll 4
          for (int lo = 0; lo < LR; ++lo) {
          const int l = LR * ql + lo;
          if (l >= D) break;
          double2 ul;
          ul.x = __shfl_sync(0xffffffffu, u[ql].x, grp * LR + lo);
          ul.y = __shfl_sync(0xffffffffu, u[ql].y, grp * LR + lo);
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            if (LR * q < D) {               // warp-uniform: some lane has a row here
              const int i = li + LR * q;
              const int ic = i < D ? i : D - 1;
              const bool low = ic >= l;
              const long long ao = low ? (long long)ic * D + l : (long long)l * D + ic;
              const double2 a = in_bounds((long long)(A - cov) + ao, (long long)nsys * D * D, kSiteSolveIn)
                                    ? __ldg(A + ao) : make_double2(0.0, 0.0);
              // R[i][l]: the conjugate above the diagonal by a sign-bit flip (a
              // negation would be one more FP64-pipe instruction per product)
              const long long flip = low ? 0LL : (long long)0x8000000000000000ull;
              const double ax = a.x,
                           ay = ic == l ? 0.0 : __longlong_as_double(__double_as_longlong(a.y) ^ flip);
              r[q].x = fma(-ax, ul.x, r[q].x);
              r[q].x = fma(ay, ul.y, r[q].x);
              r[q].y = fma(-ax, ul.y, r[q].y);
              r[q].y = fma(-ay, ul.x, r[q].y);
            }
          }
          }
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          if (LR * q < D) {
            r[q].x = fma(-delta, u[q].x, r[q].x);
            r[q].y = fma(-delta, u[q].y, r[q].y);
          }
        }
        }
        __syncwarp();
        if constexpr (F32F) {   // FP32 correction, added in FP64
          big_solve_f32<LR, RPL>(xf, Lc, rd, D, li, grp);
#pragma unroll
          for (int q = 0; q < RPL; ++q) r[q] = make_double2(xf[q].x, xf[q].y);
        } else {
          big_solve<LR, RPL>(r, Lc, rd, D, li, grp);
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          u[q].x += r[q].x;
          u[q].y += r[q].y;
        }
      }
      if (SEP) {
        if (live)
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = li + LR * q;
            if (i < D) {
              if constexpr (F32F) {   // parked in the system's weight rows as two float2
                const float4 f = to_ff4_cvt(u[q]);
                float2* park = wts + (size_t)sys * S * D + 2 * ((size_t)rhs * D + i);
                if (in_bounds((long long)(park - wts) + 1, (long long)nsys * S * D, kSiteSolveOut)) {
                  park[0] = make_float2(f.x, f.y);
                  park[1] = make_float2(f.z, f.w);
                }
              } else {
                Ubf[(size_t)rhs * D + i] = to_ff4(u[q]);
              }
            }
          }
      } else {
        emit(rsafe, u, live);
      }
    }
    if (SEP) {
      // u_s = sum_c a_s[c] U_c and its normalisation in double-float on the
      // FP32 pipe; the group's partial Re v^H u is summed in FP64
      __syncthreads();
      if constexpr (F32F) {   // the parked basis solutions over the matrix copy
        const float2* park = wts + (size_t)sys * S * D;
        for (int e = tid; e < C * D; e += NT) {
          float2 h = make_float2(0.f, 0.f), l2 = make_float2(0.f, 0.f);
          if (in_bounds((long long)(park - wts) + 2 * e + 1, (long long)nsys * S * D, kSiteSolveIn)) {
            h = park[2 * e];        // written by this CTA before the barrier: plain loads
            l2 = park[2 * e + 1];
          }
          Ubf[e] = make_float4(h.x, h.y, l2.x, l2.y);
        }
        __syncthreads();
      }
      if (prm.sym) {
        // conjugate-symmetric spatial factors (a_{S-1-s} = conj(a_s), as the
        // default steering's mirrored angles give): one pass over the basis
        // per row forms both u_s and u_{S-1-s} from four real sums,
        // P = sum ar Ur, Q = sum ai Ui, R = sum ar Ui, T = sum ai Ur:
        // u_s = (P - Q) + j (R + T), u_{S-1-s} = (P + Q) + j (R - T)
        const int npair = (S + 1) / 2;
        for (int p0 = 0; p0 < npair; p0 += NG) {
          const int pidx = p0 + g;
          const int s1 = pidx < npair ? pidx : 0;
          const int s2 = S - 1 - s1;
          const float4* as = sep_a_ff + (size_t)s1 * C;
          const float4* v1 = steer_ff + (size_t)s1 * D;
          const float4* v2 = steer_ff + (size_t)s2 * D;
          float wr1[RPL], wi1[RPL], wr2[RPL], wi2[RPL];
          ff::F2 qp1{0.f, 0.f}, qp2{0.f, 0.f};
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            wr1[q] = wi1[q] = wr2[q] = wi2[q] = 0.f;
            if (LR * q < D) {
              const int i = li + LR * q;
              const int ic = i < D ? i : D - 1;
              ff::F2 P{0.f, 0.f}, Q{0.f, 0.f}, R{0.f, 0.f}, T{0.f, 0.f};
              for (int c = 0; c < C; ++c) {
                const float4 a = __ldg(as + c);
                const float4 x = Ubf[(size_t)c * D + ic];
                const ff::F2 ar{a.x, a.y}, ai{a.z, a.w}, xr{x.x, x.y}, xi{x.z, x.w};
                P = ff::fma(P, ar, xr);
                Q = ff::fma(Q, ai, xi);
                R = ff::fma(R, ar, xi);
                T = ff::fma(T, ai, xr);
              }
              const ff::F2 ur1 = ff::sub2(P, Q), ui1 = ff::add2(R, T);
              const ff::F2 ur2 = ff::add2(P, Q), ui2 = ff::sub2(R, T);
              if (i < D) {
                const float4 a1 = __ldg(v1 + i), a2 = __ldg(v2 + i);
                qp1 = ff::fma(ff::fma(qp1, {a1.x, a1.y}, ur1), {a1.z, a1.w}, ui1);
                qp2 = ff::fma(ff::fma(qp2, {a2.x, a2.y}, ur2), {a2.z, a2.w}, ui2);
              }
              wr1[q] = __fadd_rn(ur1.hi, ur1.lo);
              wi1[q] = __fadd_rn(ui1.hi, ui1.lo);
              wr2[q] = __fadd_rn(ur2.hi, ur2.lo);
              wi2[q] = __fadd_rn(ui2.hi, ui2.lo);
            }
          }
          const double qs1 = group_sum<LR>(ff::to_double(qp1));
          const double qs2 = group_sum<LR>(ff::to_double(qp2));
          const bool good1 = ok && qs1 > 0.0 && isfinite(qs1);
          const bool good2 = ok && qs2 > 0.0 && isfinite(qs2);
          const float sf1 = good1 ? (float)rsqrt(qs1) : 0.f;
          const float sf2 = good2 ? (float)rsqrt(qs2) : 0.f;
          if (pidx < npair) {
            float2* w1 = wts + ((size_t)sys * S + s1) * D;
            float2* w2 = wts + ((size_t)sys * S + s2) * D;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
              const int i = li + LR * q;
              if (i < D) {
                if (in_bounds((long long)(w1 - wts) + i, (long long)nsys * S * D, kSiteSolveOut))
                  w1[i] = good1 ? make_float2(wr1[q] * sf1, wi1[q] * sf1) : make_float2(0.f, 0.f);
                if (s2 != s1 && in_bounds((long long)(w2 - wts) + i, (long long)nsys * S * D, kSiteSolveOut))
                  w2[i] = good2 ? make_float2(wr2[q] * sf2, wi2[q] * sf2) : make_float2(0.f, 0.f);
              }
            }
          }
        }
      } else
      for (int s0 = 0; s0 < S; s0 += NG) {
        const int s = s0 + g;
        const int ssafe = s < S ? s : 0;
        const float4* as = sep_a_ff + (size_t)ssafe * C;
        ff::F2 ur[RPL], ui[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) ur[q] = ui[q] = ff::F2{0.f, 0.f};
        for (int c = 0; c < C; ++c) {
          const float4 a = __ldg(as + c);
          const ff::F2 ar{a.x, a.y}, ai{a.z, a.w};
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            if (LR * q < D) {
              const int i = li + LR * q;
              const float4 x = Ubf[(size_t)c * D + (i < D ? i : D - 1)];
              const ff::F2 xr{x.x, x.y}, xi{x.z, x.w};
              ur[q] = ff::fms(ff::fma(ur[q], ar, xr), ai, xi);
              ui[q] = ff::fma(ff::fma(ui[q], ar, xi), ai, xr);
            }
          }
        }
        const float4* v = steer_ff + (size_t)ssafe * D;
        ff::F2 qp{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int i = li + LR * q;
          if (i < D) {
            const float4 vi = __ldg(v + i);
            qp = ff::fma(ff::fma(qp, {vi.x, vi.y}, ur[q]), {vi.z, vi.w}, ui[q]);
          }
        }
        const double qs = group_sum<LR>(ff::to_double(qp));
        const bool good = ok && qs > 0.0 && isfinite(qs);
        const float sf = good ? (float)rsqrt(qs) : 0.f;
        if (s < S) {
          float2* w = wts + ((size_t)sys * S + s) * D;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = li + LR * q;
            if (i < D)
              if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2(__fadd_rn(ur[q].hi, ur[q].lo) * sf,
                                        __fadd_rn(ui[q].hi, ui[q].lo) * sf)
                          : make_float2(0.f, 0.f);
          }
        }
      }
    }
    if (!ok && tid == 0) atomicAdd(&status->n_failed, 1ULL);
    __syncthreads();  // the next system reuses Lc, colb, Ubf, rd
  }
}

template <bool SEP, int LR, int NT, int RPL, bool F32F>
__global__ void __launch_bounds__(NT, NT >= 256 ? 1 : 3)
solve_big_kernel(SolveParams p) {
  solve_big_kernel_body<SEP, LR, NT, RPL, F32F>(p, blockIdx.x, gridDim.x);
}

// the same solves as a persistent launch over the CPIs of a batch
template <bool SEP, int LR, int NT, int RPL, bool F32F>
__global__ void __launch_bounds__(NT, NT >= 256 ? 1 : 3)
solve_big_kernel_batched(BatchCtl ctl) {
  batched_loop<SolveParams>(ctl, [&](const SolveParams& p, int bx, int, int gx) {
    solve_big_kernel_body<SEP, LR, NT, RPL, F32F>(p, bx, gx);
  });
}

// ---------------------------------------------------------------------------
// Mixed-precision iterative refinement for 32 < D <= 64 (STAP_SOLVE_MIXED_IR),
// with the layout of solve_big_kernel: one system per CTA, LR lanes per
// right-hand side holding RPL rows each.  Rl is kept in shared memory as
// double-floats (column-major packed) next to its FP32 part, which is factored
// as Lu Dg Lu^H in FP32; each right-hand side is solved in FP32 and refined
// with residuals formed from the double-float Rl by compensated (Dot2) sums on
// the FP32 pipe, the correction solved in FP32 and added to the double-float
// solution.
__host__ __device__ constexpr size_t big_mir_bytes(int D, int C, int NG, bool sep) {
  // Rl [Dp] float4, (SEP) basis solutions [C][D] float4, broadcast solutions
  // [NG][D] float4, FP32 factor [Dp] float2, pivot column [D] float2, pivot
  // reciprocals [D] float, the pivot flag and the trace
  return ((size_t)(D * (D + 1) / 2) + (sep ? (size_t)C * D : 0) + (size_t)NG * D) * 16 +
         (size_t)(D * (D + 1) / 2) * 8 + (size_t)D * 8 + ((size_t)D * 4 + 15) / 16 * 16 + 32;
}

template <bool SEP, int LR, int NT, int RPL>
__global__ void __launch_bounds__(NT)
solve_big_mir_kernel(const double2* __restrict__ cov, float2* __restrict__ wts,
                     const float4* __restrict__ steer_ff, const float4* __restrict__ g_ff,
                     const float4* __restrict__ sep_a_ff, long long nsys, int D, int S, int C,
                     double load_factor, int refine_steps, DeviceStatus* __restrict__ status) {
  extern __shared__ float4 sm4[];
  constexpr int NW = NT / 32;
  constexpr int NG = NT / LR;
  const int Dp = D * (D + 1) / 2;
  float4* Ad = sm4;                                   // [Dp] Rl, double-float, column-major
  float4* Ubf = Ad + Dp;                              // SEP: [C][D] basis solutions
  float4* uvf = Ubf + (SEP ? (size_t)C * D : 0);      // [NG][D] broadcast solutions
  float2* Lf = reinterpret_cast<float2*>(uvf + (size_t)NG * D);   // [Dp] FP32 Lu
  float2* colb = Lf + Dp;                             // [D] pivot column before division
  float* rd = reinterpret_cast<float*>(colb + D);     // [D] pivot reciprocals
  char* tail = reinterpret_cast<char*>(rd) + ((size_t)D * 4 + 15) / 16 * 16;
  int* okf = reinterpret_cast<int*>(tail);                        // pivots all positive
  double* trs = reinterpret_cast<double*>(tail + 16);             // the trace, from warp 0
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int li = lane % LR, grp = lane / LR;
  const int g = warp * (32 / LR) + grp;
  const double invD = 1.0 / (double)D;

  auto pivot = [&](float d) -> float {
    if (!(d > 0.f) || !isfinite(d)) {
      *okf = 0;
      return 1.f;
    }
    return 1.0f / d;
  };

  for (long long sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const double2* A = cov + (size_t)sys * D * D;
    if (warp == 0) {   // Re tr(R) by one warp: lanes over the diagonal, then a shuffle sum
      double tr = 0.0;
      for (int j = lane; j < D; j += 32) tr += __ldg(&A[(size_t)j * D + j].x);
      tr = group_sum<32>(tr);
      if (lane == 0) *trs = tr;
    }
    __syncthreads();
    const double delta = load_factor * *trs * invD;
    for (int i = warp; i < D; i += NW)
      for (int l = lane; l <= i; l += 32) {
        const float4 f = to_ff4_cvt(loaded(A, D, i, l, delta));
        Ad[colstart(l, D) + i - l] = f;
        Lf[colstart(l, D) + i - l] = make_float2(f.x, f.z);
      }
    __syncthreads();
    if (tid == 0) {
      *okf = 1;
      rd[0] = pivot(Lf[0].x);
    }
    __syncthreads();

    for (int j = 0; j < D; ++j) {   // FP32 Lu Dg Lu^H, as in solve_big_kernel
      const int cj = colstart(j, D);
      const float rj = rd[j];
      for (int i = j + 1 + tid; i < D; i += NT) {
        const float2 v = Lf[cj + i - j];
        colb[i] = v;
        Lf[cj + i - j] = make_float2(v.x * rj, v.y * rj);
      }
      __syncthreads();
      const int m = D - j - 1;
      const int np = m * (m + 1) / 2;
      int a = 0, off = tid;
      while (a < m && off >= m - a) off -= m - a++;
      for (int q = tid; q < np; q += NT) {
        const int l = j + 1 + a, i = l + off;
        const float2 lij = Lf[cj + i - j], alj = colb[l];
        float2 acc = Lf[colstart(l, D) + i - l];
        acc.x = fmaf(-lij.x, alj.x, acc.x);
        acc.x = fmaf(-lij.y, alj.y, acc.x);
        acc.y = fmaf(-lij.y, alj.x, acc.y);
        acc.y = fmaf(lij.x, alj.y, acc.y);
        Lf[colstart(l, D) + i - l] = acc;
        if (q == 0) rd[j + 1] = pivot(acc.x);
        off += NT;
        while (a < m && off >= m - a) off -= m - a++;
      }
      __syncthreads();
    }
    const bool ok = *okf != 0;

    const int nrhs = SEP ? C : S;
    for (int r0 = 0; r0 < nrhs; r0 += NG) {
      const int rhs = r0 + g;
      const bool live = rhs < nrhs;
      const int rsafe = live ? rhs : 0;
      auto rhs_ff = [&](int i) -> float4 {
        if (i >= D) return make_float4(0.f, 0.f, 0.f, 0.f);
        if (SEP) {
          const int t = i / C;
          return (i - t * C == rsafe) ? __ldg(g_ff + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return __ldg(steer_ff + (size_t)rsafe * D + i);
      };
      float2 x[RPL];
      ff::F2 ur[RPL], ui[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const float4 b = rhs_ff(li + LR * q);
        x[q] = make_float2(b.x, b.z);
      }
      big_solve_f32<LR, RPL>(x, Lf, rd, D, li, grp);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        ur[q] = ff::F2{x[q].x, 0.f};
        ui[q] = ff::F2{x[q].y, 0.f};
      }
      for (int it = 0; it < refine_steps; ++it) {
        // x = fl32(b - Rl u): u broadcast through shared memory, Rl[i][l]
        // from the double-float copy (conjugated above the diagonal)
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (li + LR * q < D)
            uvf[g * D + li + LR * q] = make_float4(ur[q].hi, ur[q].lo, ui[q].hi, ui[q].lo);
        __syncwarp();
        Dot2 rr[RPL], ri[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const float4 b = rhs_ff(li + LR * q);
          rr[q] = Dot2{b.x, b.y};
          ri[q] = Dot2{b.z, b.w};
        }
        // packed index of Rl[i][l]: colstart(l) + i - l below the diagonal
        // (colstart advanced incrementally), colstart(i) + l - i above
        int csi[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int i = li + LR * q;
          csi[q] = colstart(i < D ? i : D - 1, D);
        }
        int csl = 0;
        for (int l = 0; l < D; ++l) {
          const float4 ul = uvf[g * D + l];
          const ff::F2 ulr{ul.x, ul.y}, uli{ul.z, ul.w};
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            if (LR * q < D) {
              const int i = li + LR * q;
              const int ic = i < D ? i : D - 1;
              const bool low = ic >= l;
              float4 a = Ad[low ? csl + ic - l : csi[q] + l - ic];
              if (!low) {
                a.z = -a.z;
                a.w = -a.w;
              }
              dot2_cfms(rr[q], ri[q], a, ulr, uli);
            }
          }
          csl += D - l;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          x[q] = make_float2(__fadd_rn(rr[q].s, rr[q].e), __fadd_rn(ri[q].s, ri[q].e));
        big_solve_f32<LR, RPL>(x, Lf, rd, D, li, grp);
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          ur[q] = ff::add(ur[q], x[q].x);
          ui[q] = ff::add(ui[q], x[q].y);
        }
      }
      if (SEP) {
        if (live)
#pragma unroll
          for (int q = 0; q < RPL; ++q)
            if (li + LR * q < D)
              Ubf[(size_t)rhs * D + li + LR * q] = make_float4(ur[q].hi, ur[q].lo, ui[q].hi, ui[q].lo);
      } else {
        // Re v^H u over the group, the scale, the weights
        ff::F2 qp{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int i = li + LR * q;
          if (i < D) {
            const float4 v = __ldg(steer_ff + (size_t)rsafe * D + i);
            qp = ff::fma(ff::fma(qp, ff::F2{v.x, v.y}, ur[q]), ff::F2{v.z, v.w}, ui[q]);
          }
        }
        const double qs = group_sum<LR>(ff::to_double(qp));
        const bool good = ok && qs > 0.0 && isfinite(qs);
        const float sf = good ? (float)rsqrt(qs) : 0.f;
        if (live) {
          float2* w = wts + ((size_t)sys * S + rhs) * D;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = li + LR * q;
            if (i < D)
              if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2(__fadd_rn(ur[q].hi, ur[q].lo) * sf, __fadd_rn(ui[q].hi, ui[q].lo) * sf)
                          : make_float2(0.f, 0.f);
          }
        }
      }
    }
    if (SEP) {   // the combination, as in solve_big_kernel
      __syncthreads();
      for (int s0 = 0; s0 < S; s0 += NG) {
        const int s = s0 + g;
        const int ssafe = s < S ? s : 0;
        const float4* as = sep_a_ff + (size_t)ssafe * C;
        ff::F2 cr[RPL], ci[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) cr[q] = ci[q] = ff::F2{0.f, 0.f};
        for (int c = 0; c < C; ++c) {
          const float4 a = __ldg(as + c);
          const ff::F2 ar{a.x, a.y}, ai{a.z, a.w};
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            if (LR * q < D) {
              const int i = li + LR * q;
              const float4 xv = Ubf[(size_t)c * D + (i < D ? i : D - 1)];
              const ff::F2 xr{xv.x, xv.y}, xi{xv.z, xv.w};
              cr[q] = ff::fms(ff::fma(cr[q], ar, xr), ai, xi);
              ci[q] = ff::fma(ff::fma(ci[q], ar, xi), ai, xr);
            }
          }
        }
        const float4* v = steer_ff + (size_t)ssafe * D;
        ff::F2 qp{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int i = li + LR * q;
          if (i < D) {
            const float4 vi = __ldg(v + i);
            qp = ff::fma(ff::fma(qp, {vi.x, vi.y}, cr[q]), {vi.z, vi.w}, ci[q]);
          }
        }
        const double qs = group_sum<LR>(ff::to_double(qp));
        const bool good = ok && qs > 0.0 && isfinite(qs);
        const float sf = good ? (float)rsqrt(qs) : 0.f;
        if (s < S) {
          float2* w = wts + ((size_t)sys * S + s) * D;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = li + LR * q;
            if (i < D)
              if (in_bounds((long long)(w - wts) + i, (long long)nsys * S * D, kSiteSolveOut)) w[i] = good ? make_float2(__fadd_rn(cr[q].hi, cr[q].lo) * sf,
                                        __fadd_rn(ci[q].hi, ci[q].lo) * sf)
                          : make_float2(0.f, 0.f);
          }
        }
      }
    }
    if (!ok && tid == 0) atomicAdd(&status->n_failed, 1ULL);
    __syncthreads();  // the next system reuses every shared array
  }
}

template <bool SEP, int LR, int NT, int RPL>
cudaError_t launch_big_mir(const double2* cov, float2* wts, const float4* steer_ff, const float4* g_ff,
                           const float4* sep_a_ff, long long nsys, int D, int S, int C, double lf,
                           int refine, DeviceStatus* status, size_t smem, cudaStream_t s) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(solve_big_mir_kernel<SEP, LR, NT, RPL>, smem, set_bytes);
  if (e != cudaSuccess) return e;
  const int per_sm = (int)(228 * 1024 / (smem + 1024));
  long long blocks = 152LL * (per_sm < 1 ? 1 : per_sm) * 2;
  if (blocks > nsys) blocks = nsys;
  return launch_or_defer(s, [=](cudaStream_t st) {
    solve_big_mir_kernel<SEP, LR, NT, RPL><<<(unsigned)blocks, NT, smem, st>>>(
        cov, wts, steer_ff, g_ff, sep_a_ff, nsys, D, S, C, lf, refine, status);
    return cudaGetLastError();
  });
}

template <bool SEP, int LR, int NT, int RPL, bool F32F = false>
cudaError_t launch_big(const double2* cov, float2* wts, const double2* steer, const double2* sep_g,
                       const float4* steer_ff, const float4* sep_a_ff, long long nsys, int D, int S,
                       int C, double lf, int refine, DeviceStatus* status, size_t smem,
                       cudaStream_t s, bool sym = false) {
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  cudaError_t e = ensure_smem(solve_big_kernel<SEP, LR, NT, RPL, F32F>, smem, set_bytes);
  if (e == cudaSuccess) e = ensure_smem(solve_big_kernel_batched<SEP, LR, NT, RPL, F32F>, smem, set_bytes_b);
  if (e != cudaSuccess) return e;
  const int per_sm = (int)(228 * 1024 / (smem + 1024));
  long long blocks = 152LL * (per_sm < 1 ? 1 : per_sm) * 2;
  if (blocks > nsys) blocks = nsys;
  // one system per virtual block of the persistent twin
  const SolveParams p{cov, wts, steer, sep_g, nullptr, steer_ff, sep_a_ff, nsys, D, S, C, 0, lf,
                      refine, status, (int)nsys, SEP && sym ? 1 : 0};
  return launch_params(reinterpret_cast<const void*>(solve_big_kernel<SEP, LR, NT, RPL, F32F>),
                       reinterpret_cast<const void*>(solve_big_kernel_batched<SEP, LR, NT, RPL, F32F>),
                       dim3((unsigned)blocks), NT, smem, s, p, nsys);
}

template <int D, bool SEP>
cudaError_t launch_reg(const double2* cov, float2* wts, const double2* steer, const double2* sep_g,
                       const float4* steer_ff, const float4* sep_a_ff, long long nsys, int S, int C,
                       int TS, int nw, long long blocks, size_t smem, double lf, int refine,
                       DeviceStatus* status, cudaStream_t s) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  cudaError_t e = ensure_smem(solve_reg_kernel<D, SEP>, smem, set_bytes);
  if (e == cudaSuccess) e = ensure_smem(solve_reg_kernel_batched<D, SEP>, smem, set_bytes_b);
  if (e != cudaSuccess) return e;
  // one CTA's nw warps x 32/TS systems per virtual block of the persistent twin
  const long long per = (long long)nw * (32 / TS);
  const long long vb = (nsys + per - 1) / per;
  const SolveParams p{cov, wts, steer, sep_g, nullptr, steer_ff, sep_a_ff, nsys, D, S, C, TS, lf,
                      refine, status, (int)vb};
  return launch_params(reinterpret_cast<const void*>(solve_reg_kernel<D, SEP>),
                       reinterpret_cast<const void*>(solve_reg_kernel_batched<D, SEP>),
                       dim3((unsigned)blocks), nw * 32, smem, s, p, vb);
}

template <int D, bool SEP>
cudaError_t launch_mir(const double2* cov, float2* wts, const float4* steer_ff, const float4* g_ff,
                       const float4* sep_a_ff, long long nsys, int S, int C, int TS, int nw,
                       long long blocks, size_t smem, double lf, int refine, DeviceStatus* status,
                       cudaStream_t s) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static int set_bytes[64] = {0};
  cudaError_t e = ensure_smem(solve_mir_kernel<D, SEP>, smem, set_bytes);
  if (e != cudaSuccess) return e;
  return launch_or_defer(s, [=](cudaStream_t st) {
    solve_mir_kernel<D, SEP><<<(unsigned)blocks, nw * 32, smem, st>>>(
        cov, wts, steer_ff, g_ff, sep_a_ff, nsys, S, C, TS, lf, refine, status);
    return cudaGetLastError();
  });
}

}  // namespace

namespace {
__global__ void pivot_reciprocal_kernel(const double* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = recip_newton(in[i]);
}
}  // namespace

cudaError_t launch_pivot_reciprocal(const double* in, double* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  pivot_reciprocal_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

bool mir_supported(int D) { return D >= 1 && D <= kMaxD; }

namespace {

int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

cudaError_t launch_solve(const double2* cov, float2* wts, const double2* steer,
                         const double2* sep_g, const double2* sep_a, const float4* steer_ff,
                         const float4* sep_a_ff, const float4* g_ff, long long nsys, int D, int S,
                         int C, double load_factor, int refine_steps, int solver,
                         DeviceStatus* status, cudaStream_t s, const Tune& tn, bool sep_sym) {
  if (nsys <= 0) return cudaSuccess;
  if (D < 1 || D > kMaxD || S < 1) return cudaErrorInvalidValue;
  const bool sep = sep_g != nullptr && sep_a != nullptr && steer_ff != nullptr && sep_a_ff != nullptr &&
                   C >= 1 && C <= 32 && D % C == 0;
  if (solver == 1 && D > 64) {   // refinement with an FP32 factor, double-float residuals
    if (!mir_supported(D) || steer_ff == nullptr) return cudaErrorNotSupported;
    const int LR = tn.solve_lr == 16 ? 16 : 32;    // 16 lanes x 8 rows or 32 x 4, 8 warps
    const size_t Dp = (size_t)D * (D + 1) / 2;
    // FP32 factor and the two pivot columns, the double-float Rl (the basis
    // solutions' place in the combination), pivot reciprocals, pivot flag;
    // separable steering parks the C basis solutions in the S weight rows
    const size_t smem = ((Dp + 2 * D) * sizeof(float2) + 15) / 16 * 16 + Dp * 16 + D * sizeof(float) + 16;
    const bool sep_big = sep && S >= 2 * C;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
#define STAP_BIGF(lr, rpl)                                                                           \
  return sep_big ? launch_big<true, lr, 256, rpl, true>(cov, wts, steer, sep_g, steer_ff, sep_a_ff, \
                                                        nsys, D, S, C, load_factor, refine_steps,   \
                                                        status, smem, s, sep_sym)                    \
                 : launch_big<false, lr, 256, rpl, true>(cov, wts, steer, nullptr, nullptr, nullptr,\
                                                         nsys, D, S, C, load_factor, refine_steps,  \
                                                         status, smem, s)
    if (LR == 16) STAP_BIGF(16, 8);
    STAP_BIGF(32, 4);
#undef STAP_BIGF
  }
  if (solver == 1 && !(D == 8 || D == 12 || D == 16)) {  // refinement, one system per CTA
    if (!mir_supported(D) || steer_ff == nullptr) return cudaErrorNotSupported;
    const bool msep = sep && g_ff != nullptr;
    const int LR = (tn.solve_lr == 16 && D > 32) ? 16 : 8;   // 8 lanes x 8 (or 4) rows, or 16 x 4
    const int NG = 128 / LR;
    const size_t smem = big_mir_bytes(D, C, NG, msep);
    if (D <= 32)
      return msep ? launch_big_mir<true, 8, 128, 4>(cov, wts, steer_ff, g_ff, sep_a_ff, nsys, D, S, C,
                                                   load_factor, refine_steps, status, smem, s)
                  : launch_big_mir<false, 8, 128, 4>(cov, wts, steer_ff, nullptr, nullptr, nsys, D, S,
                                                    C, load_factor, refine_steps, status, smem, s);
    if (LR == 8)
      return msep ? launch_big_mir<true, 8, 128, 8>(cov, wts, steer_ff, g_ff, sep_a_ff, nsys, D, S, C,
                                                   load_factor, refine_steps, status, smem, s)
                  : launch_big_mir<false, 8, 128, 8>(cov, wts, steer_ff, nullptr, nullptr, nsys, D, S,
                                                    C, load_factor, refine_steps, status, smem, s);
    return msep ? launch_big_mir<true, 16, 128, 4>(cov, wts, steer_ff, g_ff, sep_a_ff, nsys, D, S, C,
                                                  load_factor, refine_steps, status, smem, s)
                : launch_big_mir<false, 16, 128, 4>(cov, wts, steer_ff, nullptr, nullptr, nsys, D, S, C,
                                                   load_factor, refine_steps, status, smem, s);
  }
  if (solver == 1) {  // mixed-precision iterative refinement (D = 8, 12, 16)
    if (!mir_supported(D) || steer_ff == nullptr) return cudaErrorNotSupported;
    const bool msep = sep && g_ff != nullptr;
    const int nrhs = msep ? C : S;
    int TS = pow2ceil(nrhs < 32 ? nrhs : 32);
    constexpr size_t kBudget = 200 * 1024;
    while (TS < 32 && mir_warp_bytes(D, 32 / TS, msep) * 4 > kBudget) TS <<= 1;
    if (tn.solve_ts >= TS && tn.solve_ts <= 32 && (tn.solve_ts & (tn.solve_ts - 1)) == 0)
      TS = tn.solve_ts;
    int nw = 4;
    while (nw > 1 && mir_warp_bytes(D, 32 / TS, msep) * nw > kBudget) --nw;
    if (tn.solve_nw >= 1 && tn.solve_nw <= nw) nw = tn.solve_nw;
    const size_t smem = mir_warp_bytes(D, 32 / TS, msep) * nw;
    const int G = 32 / TS;
    const long long batches = (nsys + G - 1) / G;
    long long blocks = (batches + nw - 1) / nw;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
#define STAP_MIR(d)                                                                                \
  return msep ? launch_mir<d, true>(cov, wts, steer_ff, g_ff, sep_a_ff, nsys, S, C, TS, nw, blocks, \
                                    smem, load_factor, refine_steps, status, s)                    \
              : launch_mir<d, false>(cov, wts, steer_ff, nullptr, nullptr, nsys, S, C, TS, nw,      \
                                     blocks, smem, load_factor, refine_steps, status, s)
    if (D == 8) STAP_MIR(8);
    if (D == 12) STAP_MIR(12);
    STAP_MIR(16);
#undef STAP_MIR
  }
  // one system per CTA, lanes over rows: above D = 32, and below where the
  // tuning found it faster (solve_kind 3)
  if (D > kSmallMaxD || tn.solve_kind == 3) {
    // LR lanes per right-hand side, each holding RPL rows (D <= LR * RPL):
    //   LR = 8:  RPL 8, 4 warps (D <= 64)
    //   LR = 16: RPL 4, 4 warps (D <= 64) or RPL 8, 8 warps (D <= 128)
    //   LR = 32: RPL 4, 8 warps (or 16, D > 64, when the tuning's warps per CTA is 16)
    // default: 16 up to D = 64 (several CTAs per SM), 32 above
    int LR = D <= 64 ? 16 : 32;
    if (tn.solve_lr == 32 || tn.solve_lr == 16 || (tn.solve_lr == 8 && D <= 64)) LR = tn.solve_lr;
    if (D <= kSmallMaxD) LR = 8;
    const int NT = (LR == 8 || (LR == 16 && D <= 64)) ? 128 : 256;
    const size_t Dp = (size_t)D * (D + 1) / 2;
    // Lu, the two pivot columns, (SEP) basis solutions; pivot reciprocals and the
    // pivot flag
    auto bytes = [&](bool with_u) {
      return (Dp + 2 * D) * sizeof(double2) + (with_u ? (size_t)C * D : 0) * 16 + D * sizeof(double) + 16;
    };
    const bool sep_big = sep && bytes(true) <= 227 * 1024;
    const size_t smem = bytes(sep_big);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
#define STAP_BIG(lr, nt, rpl)                                                                     \
  return sep_big ? launch_big<true, lr, nt, rpl>(cov, wts, steer, sep_g, steer_ff, sep_a_ff, nsys, D,  \
                                                 S, C, load_factor, refine_steps, status, smem, s,   \
                                                 sep_sym)                                            \
                 : launch_big<false, lr, nt, rpl>(cov, wts, steer, nullptr, nullptr, nullptr, nsys, D, \
                                                  S, C, load_factor, refine_steps, status, smem, s)
    if (LR == 8) STAP_BIG(8, 128, 8);
    if (LR == 16 && NT == 128) STAP_BIG(16, 128, 4);
    if (LR == 16) STAP_BIG(16, 256, 8);
    if (D > 64 && tn.solve_nw == 16) STAP_BIG(32, 512, 4);   // 16 warps, 16 right-hand sides at once
    STAP_BIG(32, 256, 4);
#undef STAP_BIG
  }
  constexpr size_t kBudget = 200 * 1024;
  const int Dp = D * (D + 1) / 2;
  // lanes per system: one right-hand side per lane (S steering vectors, or C
  // basis vectors when separable), more if the packed factors of 32/TS
  // systems would not fit in shared memory
  const int nrhs = sep ? C : S;
  int TS = pow2ceil(nrhs < 32 ? nrhs : 32);
  auto warp_bytes = [&](int ts) {
    const int G = 32 / ts;
    return ((size_t)G * Dp + 2 * (size_t)D * 32) * sizeof(double2) + (size_t)G * D * sizeof(double);
  };
  // register-resident kernel for D = 8, 12, 16 unless the tuning asks for the generic one
  const bool reg = (D == 8 || D == 12 || D == 16) && tn.solve_kind != 2;
  auto reg_bytes = [&](int ts) {
    const int G = 32 / ts;
    const bool alias = G * Dp >= 32 * D;
    return ((size_t)G * (Dp + D) + (sep && !alias ? (size_t)D * 32 : 0)) * sizeof(double2) +
           (size_t)G * D * sizeof(double);
  };
  if (reg) {
    while (TS < 32 && reg_bytes(TS) * 4 > kBudget) TS <<= 1;
    if (tn.solve_ts >= TS && tn.solve_ts <= 32 && (tn.solve_ts & (tn.solve_ts - 1)) == 0)
      TS = tn.solve_ts;
    int nw = 4;
    while (nw > 1 && reg_bytes(TS) * nw > kBudget) --nw;
    if (tn.solve_nw >= 1 && tn.solve_nw <= nw) nw = tn.solve_nw;
    const size_t smem = reg_bytes(TS) * nw;
    const int G = 32 / TS;
    const long long batches = (nsys + G - 1) / G;
    long long blocks = (batches + nw - 1) / nw;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    switch (D) {
      case 8: return sep ? launch_reg<8, true>(cov, wts, steer, sep_g, steer_ff, sep_a_ff, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s)
                         : launch_reg<8, false>(cov, wts, steer, nullptr, nullptr, nullptr, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s);
      case 12: return sep ? launch_reg<12, true>(cov, wts, steer, sep_g, steer_ff, sep_a_ff, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s)
                          : launch_reg<12, false>(cov, wts, steer, nullptr, nullptr, nullptr, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s);
      default: return sep ? launch_reg<16, true>(cov, wts, steer, sep_g, steer_ff, sep_a_ff, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s)
                          : launch_reg<16, false>(cov, wts, steer, nullptr, nullptr, nullptr, nsys, S, C, TS, nw, blocks, smem, load_factor, refine_steps, status, s);
    }
  }
  while (TS < 32 && warp_bytes(TS) * 4 > kBudget) TS <<= 1;
  if (tn.solve_ts >= TS && tn.solve_ts <= 32 && (tn.solve_ts & (tn.solve_ts - 1)) == 0)
    TS = tn.solve_ts;
  int nw = 4;
  while (nw > 1 && warp_bytes(TS) * nw > kBudget) --nw;
  if (tn.solve_nw >= 1 && tn.solve_nw <= nw) nw = tn.solve_nw;
  const size_t smem = warp_bytes(TS) * nw;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int G = 32 / TS;
  const long long batches = (nsys + G - 1) / G;
  long long blocks = (batches + nw - 1) / nw;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  cudaError_t e;
  // one CTA's nw warps x 32/TS systems per virtual block of the persistent twin
  const long long per = (long long)nw * G;
  const long long vb = (nsys + per - 1) / per;
  if (sep) {
    static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
    if ((e = ensure_smem(solve_kernel<true>, smem, set_bytes)) != cudaSuccess) return e;
    if ((e = ensure_smem(solve_kernel_batched<true>, smem, set_bytes_b)) != cudaSuccess) return e;
    const SolveParams p{cov, wts, steer, sep_g, sep_a, steer_ff, sep_a_ff, nsys, D, S, C, TS,
                        load_factor, refine_steps, status, (int)vb};
    return launch_params(reinterpret_cast<const void*>(solve_kernel<true>),
                         reinterpret_cast<const void*>(solve_kernel_batched<true>),
                         dim3((unsigned)blocks), nw * 32, smem, s, p, vb);
  }
  static int set_bytes[64] = {0}, set_bytes_b[64] = {0};
  if ((e = ensure_smem(solve_kernel<false>, smem, set_bytes)) != cudaSuccess) return e;
  if ((e = ensure_smem(solve_kernel_batched<false>, smem, set_bytes_b)) != cudaSuccess) return e;
  const SolveParams p{cov, wts, steer, nullptr, nullptr, nullptr, nullptr, nsys, D, S, C, TS,
                      load_factor, refine_steps, status, (int)vb};
  return launch_params(reinterpret_cast<const void*>(solve_kernel<false>),
                       reinterpret_cast<const void*>(solve_kernel_batched<false>),
                       dim3((unsigned)blocks), nw * 32, smem, s, p, vb);
}

}  // namespace stap

namespace stap {
cudaError_t check_record_solve(CheckRecord* out) { return read_check_record(out); }
}  // namespace stap
