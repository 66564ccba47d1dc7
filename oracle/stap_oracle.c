/*
 * stap_oracle.c -- plain, slow FP64 CPU oracle for the STAP hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library: it is written from
 * the definitions below and nothing else.
 *
 * What it computes (arXiv 2203.06233, Sec. 4.2 "Kernel from the STAP Signal
 * Processing Application" and Sec. 5.3 "Multi-node Results (STAP)").  The paper
 * fixes only three facts about the kernel: an explicit loop (statement S), an
 * `fft` over a 1-D domain (statement T) and a 2-D x 2-D array multiply
 * (statement U), fused into one parallel loop over data cubes.  Everything else
 * is the standard post-Doppler STAP reading, written out here step by step:
 *
 *   1. Doppler transform over pulses (statement T):
 *        h[p]       = 0.5 - 0.5 cos(2 pi p / (P-1))           symmetric Hann
 *        X[c][k][r] = sum_{p<P} h[p] x[c][p][r] exp(-j 2 pi p k / K)
 *      a direct DFT of length K >= P (zero padding), no shift, no scale.
 *   2. Space-time snapshot of cell (k, r), D = C*T entries, channel fastest:
 *        x_{k,r}[t*C + c] = X[c][(k + t - floor(T/2)) mod K][r]
 *   3. Covariance per (Doppler bin k, range block b of B cells) (statement U):
 *        R_{k,b} = (1/B) sum_{r in block b} x_{k,r} x_{k,r}^H
 *      Optional training with guard cells (not in the paper): block b's
 *      weights use the mean of R_{k,b-1} and R_{k,b+1} (oracle_train_neighbours),
 *      or, more generally, a sliding window of training groups beyond a guard
 *      band on each side of the group under test (oracle_train_window).
 *   4. Diagonal loading:  delta = lf * Re tr(R) / D,  Rl = R + delta I.
 *   5. Cholesky Rl = L L^H (L lower, real positive diagonal), column by column.
 *   6. u_s = Rl^{-1} v_s by forward then back substitution (no refinement:
 *      the FP64 solve is the reference).
 *   7. w_s = u_s / sqrt(Re v_s^H u_s)      (unit noise gain / AMF weights)
 *   8. P[s][k][r] = |w_{k,b(r),s}^H x_{k,r}|^2
 *
 *   Reduced-DOF front end (beyond the paper; oracle_reduce_channels): N
 *   element channels combined into the C channels of the cube by a matrix W.
 *
 *   PRI-staggered snapshots (an option beyond the paper; oracle_run_staggered):
 *   T sub-windows of P - T + 1 pulses replace the T adjacent bins (see the
 *   block comment above oracle_doppler_staggered).
 *
 *   Default steering (same for every Doppler bin):
 *        theta_s = -90 deg + 180 deg (s + 1/2) / S,  f_s = sin(theta_s) / 2
 *        a_c     = exp(j 2 pi f_s c)
 *        g_t     = sum_{p<P} h[p] exp(-j 2 pi m_t p / K),  m_t = t - floor(T/2)
 *        v_s[t*C + c] = g_t a_c
 *
 * All arithmetic is IEEE double (compile without -ffast-math).  Complex arrays
 * are interleaved (re, im) doubles, i.e. C99 `double complex`, row-major.
 * Range arguments (r0, nr) select a window of range cells so that very large
 * cubes can be processed a slab at a time; every step is independent across
 * range blocks, so a window that starts and ends on block boundaries gives the
 * exact result for its cells.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* The oracle's own description of one coherent processing interval. */
typedef struct {
  int32_t n_chan;          /* C */
  int32_t n_pulses;        /* P */
  int32_t n_dop;           /* K */
  int32_t n_range;         /* R */
  int32_t tdof;            /* T */
  int32_t training_block;  /* B */
  int32_t n_steering;      /* S */
} oracle_dims;

#define ORACLE_OK 0
#define ORACLE_BAD_ARGS (-1)
#define ORACLE_NO_MEMORY (-2)

static const double kPi = 3.14159265358979323846264338327950288;

static int dims_ok(const oracle_dims* d) {
  if (!d) return 0;
  if (d->n_chan < 1 || d->n_pulses < 1 || d->n_dop < d->n_pulses || d->n_range < 1) return 0;
  if (d->tdof < 1 || d->tdof > d->n_dop || d->training_block < 1 || d->n_steering < 1) return 0;
  if (d->n_range % d->training_block != 0) return 0;
  return 1;
}

static int window_ok(const oracle_dims* d, int r0, int nr) {
  return r0 >= 0 && nr >= 0 && r0 + nr <= d->n_range && r0 % d->training_block == 0 &&
         nr % d->training_block == 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Step 1 window: symmetric Hann of length P (P = 1 gives the single value 1,
 * as numpy.hanning does). */
void oracle_hann(int32_t P, double* h) {
  if (P == 1) {
    h[0] = 1.0;
    return;
  }
  for (int p = 0; p < P; ++p) h[p] = 0.5 - 0.5 * cos(2.0 * kPi * (double)p / (double)(P - 1));
}

/* exp(-j 2 pi n / K) for an integer n, with n reduced mod K exactly first. */
static cplx twiddle(int64_t n, int32_t K) {
  int64_t m = n % K;
  if (m < 0) m += K;
  double a = -2.0 * kPi * (double)m / (double)K;
  return cos(a) + I * sin(a);
}

/* Step 1 with an arbitrary real window w[P] (the Hann case is oracle_doppler).
 * cube: [C][P][R] complex (the full cube); dop: [C][K][nr] complex for the
 * range cells r0 .. r0+nr-1. */
int oracle_doppler_window(const oracle_dims* d, const double* w, const cplx* cube, int32_t r0,
                          int32_t nr, cplx* dop) {
  if (!dims_ok(d) || !w || !cube || !dop || r0 < 0 || nr < 0 || r0 + nr > d->n_range)
    return ORACLE_BAD_ARGS;
  const int C = d->n_chan, P = d->n_pulses, K = d->n_dop, R = d->n_range;
  cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)K);
  if (!tw) return ORACLE_NO_MEMORY;
  for (int n = 0; n < K; ++n) tw[n] = twiddle(n, K);
#pragma omp parallel for collapse(2) schedule(static)
  for (int c = 0; c < C; ++c) {
    for (int k = 0; k < K; ++k) {
      for (int rr = 0; rr < nr; ++rr) {
        cplx acc = 0.0;
        for (int p = 0; p < P; ++p) {
          const cplx x = cube[((size_t)c * P + p) * R + (size_t)(r0 + rr)];
          acc += w[p] * x * tw[((int64_t)p * k) % K];
        }
        dop[((size_t)c * K + k) * nr + rr] = acc;
      }
    }
  }
  free(tw);
  return ORACLE_OK;
}

int oracle_doppler(const oracle_dims* d, const cplx* cube, int32_t r0, int32_t nr, cplx* dop) {
  if (!dims_ok(d)) return ORACLE_BAD_ARGS;
  double* h = (double*)malloc(sizeof(double) * (size_t)d->n_pulses);
  if (!h) return ORACLE_NO_MEMORY;
  oracle_hann(d->n_pulses, h);
  int rc = oracle_doppler_window(d, h, cube, r0, nr, dop);
  free(h);
  return rc;
}

/* Step 2: snapshot of cell (k, rr) of a Doppler window dop[C][K][nr]. */
int oracle_snapshot(const oracle_dims* d, const cplx* dop, int32_t nr, int32_t k, int32_t rr,
                    cplx* x) {
  if (!dims_ok(d) || !dop || !x || k < 0 || k >= d->n_dop || rr < 0 || rr >= nr)
    return ORACLE_BAD_ARGS;
  const int C = d->n_chan, K = d->n_dop, T = d->tdof;
  for (int t = 0; t < T; ++t) {
    int kk = ((k + t - T / 2) % K + K) % K;
    for (int c = 0; c < C; ++c) x[t * C + c] = dop[((size_t)c * K + kk) * nr + rr];
  }
  return ORACLE_OK;
}

/* Step 3: cov[K][nr/B][D][D] from a Doppler window dop[C][K][nr]; nr must be a
 * multiple of B (the window starts on a block boundary). */
int oracle_covariance(const oracle_dims* d, const cplx* dop, int32_t nr, cplx* cov) {
  if (!dims_ok(d) || !dop || !cov || nr < 0 || nr % d->training_block != 0) return ORACLE_BAD_ARGS;
  const int K = d->n_dop, B = d->training_block, D = d->n_chan * d->tdof;
  const int NB = nr / B;
  int bad = 0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < K; ++k) {
    for (int b = 0; b < NB; ++b) {
      cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)D);
      cplx* Rm = (cplx*)calloc((size_t)D * D, sizeof(cplx));
      if (!x || !Rm) {
#pragma omp atomic write
        bad = 1;
        free(x);
        free(Rm);
        continue;
      }
      for (int rr = b * B; rr < (b + 1) * B; ++rr) {
        oracle_snapshot(d, dop, nr, k, rr, x);
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) Rm[(size_t)i * D + j] += x[i] * conj(x[j]);
      }
      cplx* out = cov + ((size_t)k * NB + b) * D * D;
      for (int i = 0; i < D * D; ++i) out[i] = Rm[i] / (double)B;
      free(x);
      free(Rm);
    }
  }
  return bad ? ORACLE_NO_MEMORY : ORACLE_OK;
}

/* Step 5: A = L L^H for Hermitian positive definite A[D][D] (only the lower
 * triangle of A is read).  L[D][D] gets the lower factor, zeros above the
 * diagonal.  Column by column: the diagonal entry from the row's squared norm,
 * then the entries below it from the inner products with earlier columns.
 * Returns 0, or 1 + the column whose pivot was not positive and finite. */
int oracle_cholesky(int32_t D, const cplx* A, cplx* L) {
  if (D < 1 || !A || !L) return ORACLE_BAD_ARGS;
  memset(L, 0, sizeof(cplx) * (size_t)D * D);
  for (int j = 0; j < D; ++j) {
    double s = creal(A[(size_t)j * D + j]);
    for (int k = 0; k < j; ++k) {
      cplx l = L[(size_t)j * D + k];
      s -= creal(l) * creal(l) + cimag(l) * cimag(l);
    }
    if (!(s > 0.0) || !isfinite(s)) return 1 + j;
    double ljj = sqrt(s);
    L[(size_t)j * D + j] = ljj;
    for (int i = j + 1; i < D; ++i) {
      cplx acc = A[(size_t)i * D + j];
      for (int k = 0; k < j; ++k) acc -= L[(size_t)i * D + k] * conj(L[(size_t)j * D + k]);
      L[(size_t)i * D + j] = acc / ljj;
    }
  }
  return ORACLE_OK;
}

/* Step 6: u = (L L^H)^{-1} b by forward substitution L y = b, then back
 * substitution L^H u = y. */
int oracle_cholesky_solve(int32_t D, const cplx* L, const cplx* b, cplx* u) {
  if (D < 1 || !L || !b || !u) return ORACLE_BAD_ARGS;
  cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)D);
  if (!y) return ORACLE_NO_MEMORY;
  for (int i = 0; i < D; ++i) {
    cplx acc = b[i];
    for (int j = 0; j < i; ++j) acc -= L[(size_t)i * D + j] * y[j];
    y[i] = acc / creal(L[(size_t)i * D + i]);
  }
  for (int i = D - 1; i >= 0; --i) {
    cplx acc = y[i];
    for (int j = i + 1; j < D; ++j) acc -= conj(L[(size_t)j * D + i]) * u[j];
    u[i] = acc / creal(L[(size_t)i * D + i]);
  }
  free(y);
  return ORACLE_OK;
}

/* Spatial part a_c of steering vector s of S: theta_s = -90 deg + 180 deg
 * (s + 1/2) / S, f_s = sin(theta_s) / 2, a_c = exp(j 2 pi f_s c). */
static cplx spatial_phase(int s, int S, int c) {
  double theta = (-90.0 + 180.0 * ((double)s + 0.5) / (double)S) * kPi / 180.0;
  double fs = 0.5 * sin(theta);
  double a = 2.0 * kPi * fs * (double)c;
  return cos(a) + I * sin(a);
}

/* Default steering table steer[S][D] (see the header comment). */
/* Temporal part g[T] of the default steering: the window's response at the
 * T bin offsets m_t = t - floor(T/2), g_t = sum_p h[p] exp(-j 2 pi m_t p / K). */
static int temporal_response(const oracle_dims* d, cplx* g) {
  const int P = d->n_pulses, K = d->n_dop, T = d->tdof;
  double* h = (double*)malloc(sizeof(double) * (size_t)P);
  if (!h) return ORACLE_NO_MEMORY;
  oracle_hann(P, h);
  for (int t = 0; t < T; ++t) {
    int m = t - T / 2;
    cplx acc = 0.0;
    for (int p = 0; p < P; ++p) acc += h[p] * twiddle((int64_t)m * p, K);
    g[t] = acc;
  }
  free(h);
  return ORACLE_OK;
}

int oracle_default_steering(const oracle_dims* d, cplx* steer) {
  if (!dims_ok(d) || !steer) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, T = d->tdof, S = d->n_steering;
  const int D = C * T;
  cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)T);
  if (!g) return ORACLE_NO_MEMORY;
  if (temporal_response(d, g) != ORACLE_OK) {
    free(g);
    return ORACLE_NO_MEMORY;
  }
  for (int s = 0; s < S; ++s)
    for (int t = 0; t < T; ++t)
      for (int c = 0; c < C; ++c) steer[(size_t)s * D + t * C + c] = g[t] * spatial_phase(s, S, c);
  free(g);
  return ORACLE_OK;
}

/* Steps 4-7 for nsys covariances cov[nsys][D][D] (lower triangle read) and a
 * steering table steer[S][D]: wts[nsys][S][D].  status[i] = 0, or 1 + the
 * failing column if system i was not positive definite (its weights are zero).
 * Returns the number of failed systems (>= 0) or a negative error. */
int oracle_weights(const oracle_dims* d, const cplx* cov, int32_t nsys, const cplx* steer,
                   double load_factor, cplx* wts, int32_t* status) {
  if (!dims_ok(d) || !cov || !steer || !wts || nsys < 0) return ORACLE_BAD_ARGS;
  const int D = d->n_chan * d->tdof, S = d->n_steering;
  int failed = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : failed)
  for (int i = 0; i < nsys; ++i) {
    const cplx* R = cov + (size_t)i * D * D;
    cplx* W = wts + (size_t)i * S * D;
    cplx* A = (cplx*)malloc(sizeof(cplx) * (size_t)D * D);
    cplx* L = (cplx*)malloc(sizeof(cplx) * (size_t)D * D);
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)D);
    if (!A || !L || !u) {
#pragma omp atomic write
      bad = 1;
      free(A);
      free(L);
      free(u);
      continue;
    }
    double tr = 0.0;
    for (int j = 0; j < D; ++j) tr += creal(R[(size_t)j * D + j]);
    const double delta = load_factor * tr / (double)D;
    memcpy(A, R, sizeof(cplx) * (size_t)D * D);
    for (int j = 0; j < D; ++j) A[(size_t)j * D + j] += delta;
    int rc = oracle_cholesky(D, A, L);
    if (status) status[i] = rc;
    if (rc != 0) {
      failed += 1;
      memset(W, 0, sizeof(cplx) * (size_t)S * D);
    } else {
      for (int s = 0; s < S; ++s) {
        const cplx* v = steer + (size_t)s * D;
        oracle_cholesky_solve(D, L, v, u);
        double q = 0.0; /* Re v^H u */
        for (int j = 0; j < D; ++j) q += creal(conj(v[j]) * u[j]);
        double scale = 1.0 / sqrt(q);
        for (int j = 0; j < D; ++j) W[(size_t)s * D + j] = u[j] * scale;
      }
    }
    free(A);
    free(L);
    free(u);
  }
  if (bad) return ORACLE_NO_MEMORY;
  return failed;
}

/* Step 8: out[S][K][nr] = |w^H x|^2 for every cell of a Doppler window
 * dop[C][K][nr] with weights wts[K][nr/B][S][D]. */
int oracle_apply(const oracle_dims* d, const cplx* dop, int32_t nr, const cplx* wts, double* out) {
  if (!dims_ok(d) || !dop || !wts || !out || nr < 0 || nr % d->training_block != 0)
    return ORACLE_BAD_ARGS;
  const int K = d->n_dop, B = d->training_block, S = d->n_steering, D = d->n_chan * d->tdof;
  const int NB = nr / B;
  int bad = 0;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < K; ++k) {
    cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)D);
    if (!x) {
#pragma omp atomic write
      bad = 1;
      continue;
    }
    for (int rr = 0; rr < nr; ++rr) {
      oracle_snapshot(d, dop, nr, k, rr, x);
      const cplx* W = wts + ((size_t)k * NB + rr / B) * S * D;
      for (int s = 0; s < S; ++s) {
        cplx y = 0.0;
        for (int j = 0; j < D; ++j) y += conj(W[(size_t)s * D + j]) * x[j];
        out[((size_t)s * K + k) * nr + rr] = creal(y) * creal(y) + cimag(y) * cimag(y);
      }
    }
    free(x);
  }
  return bad ? ORACLE_NO_MEMORY : ORACLE_OK;
}

/* Steps 1-8 for the range window [r0, r0+nr) of one CPI.  steer may be NULL
 * (default steering).  Any of dop [C][K][nr], cov [K][nr/B][D][D],
 * wts [K][nr/B][S][D] may be NULL, in which case a temporary is used; out
 * [S][K][nr] and status [K][nr/B] (may be NULL) receive the results.
 * Returns the number of failed systems or a negative error. */
int oracle_run(const oracle_dims* d, const cplx* cube, const cplx* steer, double load_factor,
               int32_t r0, int32_t nr, cplx* dop, cplx* cov, cplx* wts, double* out,
               int32_t* status) {
  if (!dims_ok(d) || !cube || !out || !window_ok(d, r0, nr)) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, K = d->n_dop, S = d->n_steering, D = d->n_chan * d->tdof;
  const int NB = nr / d->training_block;
  cplx *dop_t = NULL, *cov_t = NULL, *wts_t = NULL, *steer_t = NULL;
  int rc = ORACLE_NO_MEMORY;
  if (!dop) dop = dop_t = (cplx*)malloc(sizeof(cplx) * (size_t)C * K * nr);
  if (!cov) cov = cov_t = (cplx*)malloc(sizeof(cplx) * (size_t)K * NB * D * D);
  if (!wts) wts = wts_t = (cplx*)malloc(sizeof(cplx) * (size_t)K * NB * S * D);
  if (!steer) {
    steer = steer_t = (cplx*)malloc(sizeof(cplx) * (size_t)S * D);
    if (steer_t && oracle_default_steering(d, steer_t) != ORACLE_OK) goto done;
  }
  if (!dop || !cov || !wts || !steer) goto done;
  if ((rc = oracle_doppler(d, cube, r0, nr, dop)) != ORACLE_OK) goto done;
  if ((rc = oracle_covariance(d, dop, nr, cov)) != ORACLE_OK) goto done;
  int failed = oracle_weights(d, cov, K * NB, steer, load_factor, wts, status);
  if (failed < 0) {
    rc = failed;
    goto done;
  }
  if ((rc = oracle_apply(d, dop, nr, wts, out)) != ORACLE_OK) goto done;
  rc = failed;
done:
  free(dop_t);
  free(cov_t);
  free(wts_t);
  free(steer_t);
  return rc;
}

/* Training with guard cells (a reading beyond the paper, which trains each
 * block on its own cells): the covariance that block b's weights use is the
 * mean of the covariances of the adjacent blocks b-1 and b+1, or the one of
 * them that exists at either end of the range, so that the cell under test
 * and the other cells of its own block (its guard cells) are left out of its
 * training data.  With equal block sizes the mean of two sample covariances is
 * the sample covariance of their 2B cells.
 * cov_in: [K][nb][D][D] for nb consecutive blocks that include both ends of the
 * range where a window block has no neighbour; out: [K][nbw][D][D] for the
 * blocks b0 .. b0+nbw-1 of cov_in. */
int oracle_train_neighbours(const oracle_dims* d, const cplx* cov_in, int32_t nb, int32_t b0,
                            int32_t nbw, cplx* out) {
  if (!dims_ok(d) || !cov_in || !out || nb < 2 || b0 < 0 || nbw < 1 || b0 + nbw > nb)
    return ORACLE_BAD_ARGS;
  const int K = d->n_dop, D = d->n_chan * d->tdof;
  const size_t DD = (size_t)D * D;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < nbw; ++j) {
      const int b = b0 + j;
      const cplx* lo = b > 0 ? cov_in + ((size_t)k * nb + b - 1) * DD : NULL;
      const cplx* hi = b + 1 < nb ? cov_in + ((size_t)k * nb + b + 1) * DD : NULL;
      cplx* o = out + ((size_t)k * nbw + j) * DD;
      for (size_t e = 0; e < DD; ++e) {
        if (lo && hi) o[e] = 0.5 * (lo[e] + hi[e]);
        else o[e] = lo ? lo[e] : hi[e];
      }
    }
  return ORACLE_OK;
}

/* Steps 1-8 with the neighbour-block training above, for the window of nr
 * cells starting at cell w0 of a cube slab of d->n_range cells; the slab
 * reaches one block beyond the window on each side unless the window touches
 * that end of the range.  out: [S][K][nr]; status: [K][nr/B]. */
int oracle_run_neighbours(const oracle_dims* d, const cplx* cube, const cplx* steer,
                          double load_factor, int32_t w0, int32_t nr, double* out,
                          int32_t* status) {
  if (!dims_ok(d) || !cube || !out || !window_ok(d, w0, nr)) return ORACLE_BAD_ARGS;
  const int B = d->training_block;
  if (w0 % B != 0) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, K = d->n_dop, S = d->n_steering, D = d->n_chan * d->tdof;
  const int W = d->n_range, NBS = W / B, NBW = nr / B;
  if (NBS < 2) return ORACLE_BAD_ARGS;
  cplx* dop = (cplx*)malloc(sizeof(cplx) * (size_t)C * K * W);
  cplx* dopw = (cplx*)malloc(sizeof(cplx) * (size_t)C * K * nr);
  cplx* cov = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBS * D * D);
  cplx* trn = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBW * D * D);
  cplx* wts = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBW * S * D);
  cplx* steer_t = NULL;
  int rc = ORACLE_NO_MEMORY;
  if (!steer) {
    steer = steer_t = (cplx*)malloc(sizeof(cplx) * (size_t)S * D);
    if (steer_t && oracle_default_steering(d, steer_t) != ORACLE_OK) goto done;
  }
  if (!dop || !dopw || !cov || !trn || !wts || !steer) goto done;
  if ((rc = oracle_doppler(d, cube, 0, W, dop)) != ORACLE_OK) goto done;
  if ((rc = oracle_covariance(d, dop, W, cov)) != ORACLE_OK) goto done;
  if ((rc = oracle_train_neighbours(d, cov, NBS, w0 / B, NBW, trn)) != ORACLE_OK) goto done;
  for (int c = 0; c < C; ++c)
    for (int k = 0; k < K; ++k)
      memcpy(dopw + ((size_t)c * K + k) * nr, dop + ((size_t)c * K + k) * W + w0, sizeof(cplx) * nr);
  int failed = oracle_weights(d, trn, K * NBW, steer, load_factor, wts, status);
  if (failed < 0) {
    rc = failed;
    goto done;
  }
  if ((rc = oracle_apply(d, dopw, nr, wts, out)) != ORACLE_OK) goto done;
  rc = failed;
done:
  free(dop);
  free(dopw);
  free(cov);
  free(trn);
  free(wts);
  free(steer_t);
  return rc;
}

/* Sliding training window with guard cells (a reading beyond the paper,
 * which trains each block on its own cells; it generalises the neighbour-block
 * training above).  The range axis is cut into groups of B cells (B = 1: each
 * cell is its own group, i.e. a per-cell window); group j's weights come from
 * the training groups
 *   T(j) = { j-guard-half, ..., j-guard-1 }  u  { j+guard+1, ..., j+guard+half }
 * that exist in 0 .. nb-1: `guard` groups on each side of j (and j itself)
 * are guard cells, left out of j's training data, and `half` groups on each
 * side beyond them train it.  Near the ends of the range the groups that do
 * not exist are dropped.  The training covariance is the mean of the groups'
 * covariances, summed left side first, in increasing group order:
 *   R_train(j) = (1 / |T(j)|) sum_{i in T(j)} R_{k,i}
 * which with equal group sizes is the sample covariance of all the training
 * cells.  guard = 0, half = 1 is the neighbour-block training.  Needs
 * half >= 1, guard >= 0 and nb >= 2 guard + 2 (then every group has
 * training groups on at least one side).
 * cov_in: [K][nb][D][D] for nb consecutive groups that include every group
 * that trains a window group; out: [K][nbw][D][D] for the groups
 * b0 .. b0+nbw-1 of cov_in. */
int oracle_train_window(const oracle_dims* d, const cplx* cov_in, int32_t nb, int32_t b0,
                        int32_t nbw, int32_t guard, int32_t half, cplx* out) {
  if (!dims_ok(d) || !cov_in || !out || guard < 0 || half < 1 || nb < 2 * guard + 2 || b0 < 0 ||
      nbw < 1 || b0 + nbw > nb)
    return ORACLE_BAD_ARGS;
  const int K = d->n_dop, D = d->n_chan * d->tdof;
  const size_t DD = (size_t)D * D;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < K; ++k)
    for (int jw = 0; jw < nbw; ++jw) {
      const int j = b0 + jw;
      cplx* o = out + ((size_t)k * nbw + jw) * DD;
      for (size_t e = 0; e < DD; ++e) o[e] = 0.0;
      int count = 0;
      for (int side = 0; side < 2; ++side)
        for (int m = 0; m < half; ++m) {
          const int i = side == 0 ? j - guard - half + m : j + guard + 1 + m;
          if (i < 0 || i >= nb) continue;
          const cplx* in = cov_in + ((size_t)k * nb + i) * DD;
          for (size_t e = 0; e < DD; ++e) o[e] += in[e];
          ++count;
        }
      for (size_t e = 0; e < DD; ++e) o[e] /= (double)count;
    }
  return ORACLE_OK;
}

/* Steps 1-8 with the sliding training window above, for the window of nr
 * cells starting at cell w0 of a cube slab of d->n_range cells; the slab
 * reaches (guard + half) groups beyond the window on each side unless the
 * window touches that end of the range (the slab then starts or ends there).
 * out: [S][K][nr]; status: [K][nr/B]. */
int oracle_run_window(const oracle_dims* d, const cplx* cube, const cplx* steer, double load_factor,
                      int32_t w0, int32_t nr, int32_t guard, int32_t half, double* out,
                      int32_t* status) {
  if (!dims_ok(d) || !cube || !out || !window_ok(d, w0, nr)) return ORACLE_BAD_ARGS;
  const int B = d->training_block;
  if (w0 % B != 0) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, K = d->n_dop, S = d->n_steering, D = d->n_chan * d->tdof;
  const int W = d->n_range, NBS = W / B, NBW = nr / B;
  if (guard < 0 || half < 1 || NBS < 2 * guard + 2) return ORACLE_BAD_ARGS;
  cplx* dop = (cplx*)malloc(sizeof(cplx) * (size_t)C * K * W);
  cplx* dopw = (cplx*)malloc(sizeof(cplx) * (size_t)C * K * nr);
  cplx* cov = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBS * D * D);
  cplx* trn = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBW * D * D);
  cplx* wts = (cplx*)malloc(sizeof(cplx) * (size_t)K * NBW * S * D);
  cplx* steer_t = NULL;
  int rc = ORACLE_NO_MEMORY;
  if (!steer) {
    steer = steer_t = (cplx*)malloc(sizeof(cplx) * (size_t)S * D);
    if (steer_t && oracle_default_steering(d, steer_t) != ORACLE_OK) goto done;
  }
  if (!dop || !dopw || !cov || !trn || !wts || !steer) goto done;
  if ((rc = oracle_doppler(d, cube, 0, W, dop)) != ORACLE_OK) goto done;
  if ((rc = oracle_covariance(d, dop, W, cov)) != ORACLE_OK) goto done;
  if ((rc = oracle_train_window(d, cov, NBS, w0 / B, NBW, guard, half, trn)) != ORACLE_OK) goto done;
  for (int c = 0; c < C; ++c)
    for (int k = 0; k < K; ++k)
      memcpy(dopw + ((size_t)c * K + k) * nr, dop + ((size_t)c * K + k) * W + w0, sizeof(cplx) * nr);
  int failed = oracle_weights(d, trn, K * NBW, steer, load_factor, wts, status);
  if (failed < 0) {
    rc = failed;
    goto done;
  }
  if ((rc = oracle_apply(d, dopw, nr, wts, out)) != ORACLE_OK) goto done;
  rc = failed;
done:
  free(dop);
  free(dopw);
  free(cov);
  free(trn);
  free(wts);
  free(steer_t);
  return rc;
}

/* ---------------------------------------------------------------------------
 * PRI-staggered post-Doppler (a variant beyond the paper's kernel, which fixes
 * only an fft over pulses): the T temporal degrees of freedom come from T
 * sub-windows of P' = P - T + 1 consecutive pulses instead of T adjacent bins
 * of one transform.  Sub-window t holds the pulses t .. t+P'-1, windowed by the
 * symmetric Hann h' of length P'; each pulse keeps the phase of its index in
 * the whole CPI:
 *   Xs[t][c][k][r] = sum_{p=t}^{t+P'-1} h'[p - t] x[c][p][r] exp(-j 2 pi p k / K)
 * The snapshot of cell (k, r) takes the same bin of every sub-window,
 *   x_{k,r}[t*C + c] = Xs[t][c][k][r],
 * so Xs[T][C][K][R] is a Doppler cube of C*T channels with one bin per
 * snapshot, and steps 3-8 are the ones above for the dims (C*T, P, K, R, 1, B,
 * S).  A unit target at bin centre k/K and angle theta_s gives
 * Xs[t][c][k] = G a_c in every sub-window (G = sum h'), hence the steering
 *   v_s[t*C + c] = G a_c.
 * Referencing each sub-window to its own first pulse instead multiplies
 * sub-window t's bin k by exp(j 2 pi k t / K) and the steering by the same
 * factor; that diagonal unitary change of basis leaves every output power
 * unchanged.
 */

/* The dims under which steps 3-8 see the staggered snapshots. */
static oracle_dims staggered_inner(const oracle_dims* d) {
  oracle_dims e = *d;
  e.n_chan = d->n_chan * d->tdof;
  e.tdof = 1;
  return e;
}

static int staggered_ok(const oracle_dims* d) {
  return dims_ok(d) && d->tdof <= d->n_pulses;
}

/* dop[T][C][K][nr] for the range cells r0 .. r0+nr-1 of cube[C][P][R]. */
int oracle_doppler_staggered(const oracle_dims* d, const cplx* cube, int32_t r0, int32_t nr,
                             cplx* dop) {
  if (!staggered_ok(d) || !cube || !dop || r0 < 0 || nr < 0 || r0 + nr > d->n_range)
    return ORACLE_BAD_ARGS;
  const int C = d->n_chan, P = d->n_pulses, K = d->n_dop, R = d->n_range, T = d->tdof;
  const int Ps = P - T + 1;
  double* h = (double*)malloc(sizeof(double) * (size_t)Ps);
  cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)K);
  if (!h || !tw) {
    free(h);
    free(tw);
    return ORACLE_NO_MEMORY;
  }
  oracle_hann(Ps, h);
  for (int n = 0; n < K; ++n) tw[n] = twiddle(n, K);
#pragma omp parallel for collapse(3) schedule(static)
  for (int t = 0; t < T; ++t) {
    for (int c = 0; c < C; ++c) {
      for (int k = 0; k < K; ++k) {
        for (int rr = 0; rr < nr; ++rr) {
          cplx acc = 0.0;
          for (int p = t; p < t + Ps; ++p) {
            const cplx x = cube[((size_t)c * P + p) * R + (size_t)(r0 + rr)];
            acc += h[p - t] * x * tw[((int64_t)p * k) % K];
          }
          dop[(((size_t)t * C + c) * K + k) * nr + rr] = acc;
        }
      }
    }
  }
  free(h);
  free(tw);
  return ORACLE_OK;
}

/* Default steering steer[S][D] of the staggered snapshots (same for every bin). */
int oracle_default_steering_staggered(const oracle_dims* d, cplx* steer) {
  if (!staggered_ok(d) || !steer) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, T = d->tdof, S = d->n_steering, D = C * T;
  const int Ps = d->n_pulses - T + 1;
  double* h = (double*)malloc(sizeof(double) * (size_t)Ps);
  if (!h) return ORACLE_NO_MEMORY;
  oracle_hann(Ps, h);
  double G = 0.0;
  for (int p = 0; p < Ps; ++p) G += h[p];
  for (int s = 0; s < S; ++s)
    for (int t = 0; t < T; ++t)
      for (int c = 0; c < C; ++c) steer[(size_t)s * D + t * C + c] = G * spatial_phase(s, S, c);
  free(h);
  return ORACLE_OK;
}

/* Steps 1-8 with the staggered transform, as oracle_run: dop [T][C][K][nr],
 * cov [K][nr/B][D][D], wts [K][nr/B][S][D] (each may be NULL), out [S][K][nr]. */
int oracle_run_staggered(const oracle_dims* d, const cplx* cube, const cplx* steer,
                         double load_factor, int32_t r0, int32_t nr, cplx* dop, cplx* cov,
                         cplx* wts, double* out, int32_t* status) {
  if (!staggered_ok(d) || !cube || !out || !window_ok(d, r0, nr)) return ORACLE_BAD_ARGS;
  const oracle_dims e = staggered_inner(d);
  const int K = d->n_dop, S = d->n_steering, D = d->n_chan * d->tdof;
  const int NB = nr / d->training_block;
  cplx *dop_t = NULL, *cov_t = NULL, *wts_t = NULL, *steer_t = NULL;
  int rc = ORACLE_NO_MEMORY;
  if (!dop) dop = dop_t = (cplx*)malloc(sizeof(cplx) * (size_t)D * K * nr);
  if (!cov) cov = cov_t = (cplx*)malloc(sizeof(cplx) * (size_t)K * NB * D * D);
  if (!wts) wts = wts_t = (cplx*)malloc(sizeof(cplx) * (size_t)K * NB * S * D);
  if (!steer) {
    steer = steer_t = (cplx*)malloc(sizeof(cplx) * (size_t)S * D);
    if (steer_t && oracle_default_steering_staggered(d, steer_t) != ORACLE_OK) goto done;
  }
  if (!dop || !cov || !wts || !steer) goto done;
  if ((rc = oracle_doppler_staggered(d, cube, r0, nr, dop)) != ORACLE_OK) goto done;
  if ((rc = oracle_covariance(&e, dop, nr, cov)) != ORACLE_OK) goto done;
  int failed = oracle_weights(&e, cov, K * NB, steer, load_factor, wts, status);
  if (failed < 0) {
    rc = failed;
    goto done;
  }
  if ((rc = oracle_apply(&e, dop, nr, wts, out)) != ORACLE_OK) goto done;
  rc = failed;
done:
  free(dop_t);
  free(cov_t);
  free(wts_t);
  free(steer_t);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Reduced-DOF front end (a step beyond the paper, whose 1000-channel cubes
 * would make D = 1000 T): the N element channels of an element cube
 * x[N][P][R] (a half-wavelength line array, element n at phase
 * exp(j 2 pi f n) for spatial frequency f) are combined into the C channels
 * of the STAP cube by a matrix W[C][N]:
 *   y[c][p][r] = sum_{n<N} conj(W[c][n]) x[n][p][r].
 * The default W sums C contiguous subarrays of N / C elements (N a multiple of
 * C).  A plane wave at spatial frequency f_s reaches channel c with gain
 *   b_s[c] = sum_n conj(W[c][n]) exp(j 2 pi f_s n),
 * so the steering of the reduced snapshots is v_s[t*C + c] = g_t b_s[c]
 * (g as in the default steering); steps 1-8 then run unchanged on y.
 */

/* y[C][P][R] from x[N][P][R] and W[C][N]. */
int oracle_reduce_channels(int32_t N, int32_t C, int32_t P, int32_t R, const cplx* W,
                           const cplx* x, cplx* y) {
  if (N < 1 || C < 1 || P < 1 || R < 1 || !W || !x || !y) return ORACLE_BAD_ARGS;
#pragma omp parallel for collapse(2) schedule(static)
  for (int c = 0; c < C; ++c)
    for (int p = 0; p < P; ++p)
      for (int r = 0; r < R; ++r) {
        cplx acc = 0.0;
        for (int n = 0; n < N; ++n)
          acc += conj(W[(size_t)c * N + n]) * x[((size_t)n * P + p) * R + r];
        y[((size_t)c * P + p) * R + r] = acc;
      }
  return ORACLE_OK;
}

/* W[C][N] of C contiguous subarrays: 1 for c N/C <= n < (c+1) N/C, else 0. */
int oracle_subarray_weights(int32_t N, int32_t C, cplx* W) {
  if (N < 1 || C < 1 || N % C != 0 || !W) return ORACLE_BAD_ARGS;
  const int M = N / C;
  for (int c = 0; c < C; ++c)
    for (int n = 0; n < N; ++n) W[(size_t)c * N + n] = (n / M == c) ? 1.0 : 0.0;
  return ORACLE_OK;
}

/* Steering steer[S][D] of snapshots of the reduced channels (d->n_chan = C). */
int oracle_reduced_steering(const oracle_dims* d, int32_t N, const cplx* W, cplx* steer) {
  if (!dims_ok(d) || N < 1 || !W || !steer) return ORACLE_BAD_ARGS;
  const int C = d->n_chan, T = d->tdof, S = d->n_steering;
  const int D = C * T;
  cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)T);
  cplx* b = (cplx*)malloc(sizeof(cplx) * (size_t)C);
  if (!g || !b || temporal_response(d, g) != ORACLE_OK) {
    free(g);
    free(b);
    return ORACLE_NO_MEMORY;
  }
  for (int s = 0; s < S; ++s) {
    for (int c = 0; c < C; ++c) {
      cplx acc = 0.0;
      for (int n = 0; n < N; ++n) acc += conj(W[(size_t)c * N + n]) * spatial_phase(s, S, n);
      b[c] = acc;
    }
    for (int t = 0; t < T; ++t)
      for (int c = 0; c < C; ++c) steer[(size_t)s * D + t * C + c] = g[t] * b[c];
  }
  free(g);
  free(b);
  return ORACLE_OK;
}
