/*
 * stap.h -- C ABI of libstap, a GB300 (sm_103a) implementation of the
 * Space-Time Adaptive Processing (STAP) radar kernel.
 *
 * The operation is the STAP kernel of arXiv 2203.06233, Sec. 4.2 (the kernel
 * figure: an explicit loop, statement S; an `fft` over a 1-D domain, statement
 * T; a 2-D x 2-D array multiply, statement U; all fused into one parallel loop
 * over data cubes) and Sec. 5.3 (the STAP workload: data cubes of pulses x
 * channels x range samples, throughput in cubes per second).  The paper gives
 * no formulas; each call below states the post-Doppler reading it implements.
 *
 * Notation: C channels, P pulses, K Doppler bins (K >= P), R range cells,
 * T adjacent-bin degrees of freedom, D = C*T snapshot length, B cells per
 * training block, NB = R/B blocks, S steering vectors.
 *
 * Conventions shared by every call:
 *  - Buffers are DEVICE pointers owned by the caller, 16-byte aligned, dense
 *    row-major in the layout given.  Complex values are interleaved (re, im):
 *    "c64" = 2 x float, "c128" = 2 x double.
 *  - Calls are asynchronous on the plan's CUDA stream.  Argument, shape and
 *    alignment errors are returned synchronously and launch nothing.  Errors
 *    found on the device (a covariance that is not positive definite) are
 *    counted in the workspace and read back by stap_get_status.
 *  - No call allocates device memory.  Scratch comes from the caller through
 *    stap_plan_set_workspace; its contents between calls belong to the plan.
 *  - No exception crosses the ABI.  A plan is not thread-safe: one host thread
 *    at a time per plan.
 */
#ifndef STAP_H_
#define STAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STAP_ABI_VERSION 5

typedef enum {
  STAP_OK = 0,
  STAP_ERR_INVALID_ARG = 1,  /* NULL pointer, bad option value, wrong CPI index */
  STAP_ERR_SHAPE = 2,        /* dims violate K >= P, R % B == 0, 1 <= T <= K, ... */
  STAP_ERR_UNSUPPORTED = 3,  /* valid STAP shape outside what the kernels handle */
  STAP_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
  STAP_ERR_NOT_POSDEF = 5,   /* some loaded covariances were not positive definite */
  STAP_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  STAP_ERR_NO_WORKSPACE = 7, /* workspace missing or smaller than the call needs */
  STAP_ERR_MISALIGNED = 8    /* a buffer is not 16-byte aligned */
} stap_status;

/* Arithmetic of the contraction steps (Doppler, covariance, apply).  The
 * factorisation and the triangular solves follow stap_solver.  The mixed
 * precisions put the covariance (statement U, Sec. 4.2) and the apply on the
 * tensor cores as split products with FP32 accumulation; the Doppler
 * transform stays the FP32 FFT.  Each product of two values is formed from
 * pieces that the values are split into:
 *   TF32X3       x = hi + lo (TF32); hi*hi + hi*lo + lo*hi: about 2^-21
 *                relative per product;
 *   BF16X3       x = hi + mid + lo (BF16, each the rounding of what the
 *                earlier pieces leave); the six products of pieces whose
 *                orders sum to at most 2: about 2^-24 relative per product;
 *   FP16_SCALED  per-block scaling: every value of a block (one covariance
 *                system, i.e. one Doppler bin and range block; the snapshots
 *                of one 128-cell apply tile; one weight vector) is multiplied
 *                by the power of two that brings the block's largest
 *                magnitude into [2^14, 2^15); then x 2^e = hi + lo (FP16);
 *                hi*hi + hi*lo + lo*hi, the scales removed exactly afterwards:
 *                about 2^-21 relative to the block's largest magnitude.
 * The tensor-core apply needs B | 128 or 128 | B and at most 256 real weight
 * rows (2 per steering vector and block) per 128-cell tile, and falls back
 * to the FP32 apply otherwise; stap_plan_autotune keeps the FP32 kernel of a
 * step where that is faster (small D). */
typedef enum {
  STAP_PREC_FP32 = 0,        /* FP32 FFT; covariance accumulated error-free in
                                FP32 pairs (two-product / compensated sum); FP32
                                apply */
  STAP_PREC_BF16X3 = 1,      /* mixed: BF16 three-piece split, 6 products */
  STAP_PREC_TF32X3 = 2,      /* mixed: TF32 two-piece split, 3 products */
  STAP_PREC_FP16_SCALED = 3  /* mixed: FP16 two-piece split with per-block
                                power-of-two scaling, 3 products */
} stap_precision;

/* Arithmetic of the weight solve (diagonal load, factorisation, substitutions,
 * refinement). */
typedef enum {
  STAP_SOLVE_FP64 = 0,    /* FP64 factorisation and substitutions; each of the
                             refine_steps refinement steps forms the FP64
                             residual v - Rl u and solves for the correction in
                             FP64 (the default) */
  STAP_SOLVE_MIXED_IR = 1 /* mixed-precision iterative refinement (not in the
                             paper; a faster option): Rl split into
                             double-floats (hi + lo, about 2^-48), its FP32 part
                             factored and solved in FP32, and each of the
                             refine_steps steps forms the residual v - Rl u in
                             double-float arithmetic on the FP32 pipe, solves
                             for the correction in FP32 and adds it to the
                             double-float solution.  Each step shrinks the error
                             by about cond(Rl) 2^-24; 2 steps reach FP32 weight
                             accuracy for cond(Rl) up to about 1e5.  For
                             D > 64 the residual is formed in FP64 from the
                             input instead (the double-float matrix would not
                             fit on chip) */
} stap_solver;

/* Which range cells train the covariance that block b's weights use. */
typedef enum {
  STAP_TRAIN_OWN_BLOCK = 0,      /* the B cells of block b itself, the cell under
                                    test included (the default) */
  STAP_TRAIN_NEIGHBOURS = 1,     /* not in the paper: the blocks b-1 and b+1 (the
                                    one that exists at either end of the range),
                                    i.e. the cell under test and the other cells
                                    of its block are guard cells; needs NB >= 2.
                                    One-CPI runs are then not cut into range
                                    slabs (block b needs its neighbours' data) */
  STAP_TRAIN_WINDOW = 2          /* not in the paper: a sliding window with a
                                    guard band.  The range axis is cut into groups
                                    of B = training_block cells (B = 1: a window
                                    per cell); group j's weights come from the
                                    covariances of the groups
                                      j-g-h .. j-g-1  and  j+g+1 .. j+g+h
                                    that exist (g = train_guard guard groups on
                                    each side, h = train_half training groups
                                    beyond them), averaged, i.e. the sample
                                    covariance of those h B .. 2 h B cells.  The
                                    cell under test, its group and g groups on
                                    each side are left out of its training.
                                    g = 0, h = 1 is STAP_TRAIN_NEIGHBOURS.  Needs
                                    NB >= 2 g + 2.  One-CPI runs are not cut into
                                    range slabs */
} stap_training;

/* Where a snapshot's T temporal degrees of freedom come from. */
typedef enum {
  STAP_SNAP_ADJACENT_BINS = 0, /* T adjacent bins of one Doppler transform of all
                                  P pulses (the default) */
  STAP_SNAP_PRI_STAGGERED = 1  /* not in the paper: T transforms of P' = P - T + 1
                                  pulses each, sub-window t starting at pulse t,
                                  windowed by the symmetric Hann of length P' and
                                  keeping each pulse's CPI phase:
                                    Xs[t][c][k][r] = sum_{p=t}^{t+P'-1}
                                      h'[p-t] cube[c][p][r] exp(-j 2 pi p k / K);
                                  the snapshot of bin k takes bin k of every
                                  sub-window.  The Doppler output then has C*T
                                  rows (row t*C + c); needs T <= P */
} stap_snapshots;

typedef struct {
  int32_t n_chan;         /* C >= 1 */
  int32_t n_pulses;       /* P >= 1 */
  int32_t n_dop;          /* K >= P, a power of two, K <= 1024 */
  int32_t n_range;        /* R >= 1, a multiple of B */
  int32_t tdof;           /* 1 <= T <= K; D = n_chan * tdof <= 128 */
  int32_t training_block; /* B >= 1 */
  int32_t n_steering;     /* S >= 1 */
} stap_dims;

typedef struct {
  double load_factor;   /* diagonal load delta = load_factor * Re tr(R) / D; >= 0 (default 1e-3) */
  int32_t refine_steps; /* iterative-refinement steps after the first solve, 0..4 (default 1) */
  int32_t precision;    /* a stap_precision value (default STAP_PREC_FP32) */
  int32_t solver;       /* a stap_solver value (default STAP_SOLVE_FP64) */
  int32_t training;     /* a stap_training value (default STAP_TRAIN_OWN_BLOCK) */
  int32_t snapshots;    /* a stap_snapshots value (default STAP_SNAP_ADJACENT_BINS) */
  int32_t train_guard;  /* STAP_TRAIN_WINDOW: guard groups on each side, >= 0 (default 0) */
  int32_t train_half;   /* STAP_TRAIN_WINDOW: training groups on each side, >= 1 (default 1) */
} stap_options;

typedef struct stap_plan_s* stap_plan;

/* Fill *opt with the defaults (load_factor 1e-3, refine_steps 1, FP32, FP64
 * solve, own-block training, adjacent-bin snapshots, train_guard 0,
 * train_half 1). */
void stap_options_default(stap_options* opt);

/* Create a plan for n_cpi CPIs whose shapes are dims[0 .. n_cpi-1].
 * opt may be NULL (defaults).  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream).  On success *out is the plan and, if workspace_bytes is not
 * NULL, *workspace_bytes the device workspace stap_run_cpi needs (the
 * step-by-step calls need less, see stap_plan_workspace_sizes).  Host-only:
 * makes no CUDA call.  Sets the default steering table of every CPI:
 *   theta_s = -90 + 180 (s + 1/2)/S degrees, f_s = sin(theta_s)/2,
 *   a_c = exp(j 2 pi f_s c),  g_t = sum_p h[p] exp(-j 2 pi (t - floor(T/2)) p / K),
 *   v_s[t*C + c] = g_t a_c   (h = symmetric Hann of length P).
 * With STAP_SNAP_PRI_STAGGERED, g_t = sum_p h'[p] for every t (a target at a
 * bin centre has the same response in every sub-window). */
stap_status stap_plan_create(const stap_dims* dims, int32_t n_cpi, const stap_options* opt,
                             void* cuda_stream, stap_plan* out, size_t* workspace_bytes);

/* step_bytes: workspace needed by the step-by-step calls (tables and status);
 * run_bytes: workspace needed by stap_run_cpi (adds the intermediates of the
 * largest CPI).  Either pointer may be NULL. */
stap_status stap_plan_workspace_sizes(stap_plan plan, size_t* step_bytes, size_t* run_bytes);

/* Hand the plan a device workspace of `bytes` bytes (16-byte aligned, caller-
 * owned, kept until destroy or the next call of this function).  Uploads the
 * plan's tables on the plan's stream and clears the device status. */
stap_status stap_plan_set_workspace(stap_plan plan, void* dev_ptr, size_t bytes);

/* Polls of an mbarrier after which a pipeline wait of the tensor-core
 * kernels (STAP_PREC_TF32X3 covariance and apply) gives up, by default
 * STAP_DEFAULT_WAIT_POLLS.  A CTA whose wait gave up records a timeout (read
 * by stap_get_status as STAP_ERR_TIMEOUT), waits for the tensor-core
 * operations it has in flight (those waits always use the default limit),
 * frees its tensor memory and exits; that launch's outputs are then
 * incomplete.  0 makes every pipeline wait give up at once, which exercises
 * this path on a healthy GPU.  No counterpart in the paper (failure
 * detection of the device code).  STAP_ERR_INVALID_ARG if max_polls < 0.
 * Drops a captured batch graph. */
#define STAP_DEFAULT_WAIT_POLLS 4194304
stap_status stap_plan_set_wait_limit(stap_plan plan, int32_t max_polls);

/* Change the stream later calls are issued on. */
stap_status stap_plan_set_stream(stap_plan plan, void* cuda_stream);

/* Replace the steering table of CPI `cpi` with host_c128[S][D] (copied).
 * Needs the workspace to be set (the table is uploaded on the plan's stream). */
stap_status stap_plan_set_steering(stap_plan plan, int32_t cpi, const double* host_c128);

stap_status stap_plan_destroy(stap_plan plan);

/* Statement T (Sec. 4.2): Hann-windowed DFT over pulses, zero-padded to K.
 *   dop[c][k][r] = sum_{p<P} h[p] cube[c][p][r] exp(-j 2 pi p k / K)
 * cube: c64 [C][P][R]; dop: c64 [C][K][R].  With STAP_SNAP_PRI_STAGGERED:
 * dop[t*C + c][k][r] = Xs[t][c][k][r] (see stap_snapshots), c64 [C*T][K][R].
 * Single-CPI plans only. */
stap_status stap_doppler(stap_plan plan, const void* cube_c64, void* dop_c64);

/* Statement U (Sec. 4.2), one covariance per (Doppler bin k, range block b):
 *   x_{k,r}[t*C + c] = dop[c][(k + t - floor(T/2)) mod K][r]
 *   cov[k][b] = (1/B) sum_{r = bB}^{bB+B-1} x_{k,r} x_{k,r}^H
 * dop: c64 [C][K][R]; cov: c128 [K][NB][D][D], full Hermitian.
 * With STAP_SNAP_PRI_STAGGERED: x_{k,r}[t*C + c] = dop[t*C + c][k][r], dop
 * c64 [C*T][K][R]. */
stap_status stap_covariance(stap_plan plan, const void* dop_c64, void* cov_c128);

/* Training matrices for STAP_TRAIN_NEIGHBOURS, from the per-block covariances
 * of stap_covariance:
 *   cov_train[k][b] = (cov[k][b-1] + cov[k][b+1]) / 2, or the one of them
 *   that exists for b = 0 and b = NB-1.
 * cov, cov_train: c128 [K][NB][D][D], distinct buffers.  stap_run_cpi applies
 * it between the covariance and the solve when the plan's training is
 * STAP_TRAIN_NEIGHBOURS; step-by-step callers pass cov_train to
 * stap_solve_weights themselves.  STAP_ERR_SHAPE if NB < 2. */
stap_status stap_train_neighbours(stap_plan plan, const void* cov_c128, void* cov_train_c128);

/* Training matrices of the sliding window (STAP_TRAIN_WINDOW, with the
 * plan's train_guard g and train_half h; other plans use g = 0, h = 1, the
 * neighbour-block form), from the per-group covariances of stap_covariance:
 *   cov_train[k][j] = mean of cov[k][i] over the groups i in
 *                     j-g-h .. j-g-1 and j+g+1 .. j+g+h with 0 <= i < NB,
 * summed left side first in increasing i, each component then divided by
 * the count.  cov, cov_train: c128 [K][NB][D][D], distinct buffers.
 * stap_run_cpi applies it between the covariance and the solve when the
 * plan's training is STAP_TRAIN_WINDOW.  STAP_ERR_SHAPE if NB < 2 g + 2. */
stap_status stap_train_window(stap_plan plan, const void* cov_c128, void* cov_train_c128);

/* Adaptive weights per (k, b) and steering vector v_s (Sec. 4.2's STAP
 * kernel, loaded sample-matrix reading), in FP64 with the default solver:
 *   delta = load_factor * Re tr(cov) / D,  Rl = cov + delta I = L L^H,
 *   u_s = Rl^{-1} v_s by forward/back substitution, refine_steps refinement
 *   steps u_s += Rl^{-1} (v_s - Rl u_s),  w_s = u_s / sqrt(Re v_s^H u_s).
 * (STAP_SOLVE_MIXED_IR: see stap_solver.)
 * Only the lower triangle and the real part of the diagonal of each cov are
 * read.  A system whose pivot is not positive and finite gets zero weights
 * and is counted (stap_get_status).  cov: c128 [K][NB][D][D];
 * wts: c64 [K][NB][S][D]. */
stap_status stap_solve_weights(stap_plan plan, const void* cov_c128, void* wts_c64);

/* Output power of every range-Doppler cell:
 *   out[s][k][r] = | w_{k, r/B, s}^H x_{k,r} |^2
 * dop: c64 [C][K][R] (STAP_SNAP_PRI_STAGGERED: [C*T][K][R], snapshots as in
 * stap_covariance); wts: c64 [K][NB][S][D]; out: float [S][K][R]. */
stap_status stap_apply(stap_plan plan, const void* dop_c64, const void* wts_c64, float* out);

/* The whole chain (Doppler, covariance, weights, apply) for every CPI of the
 * plan, with the intermediates in the workspace and no host round trip.
 * cubes[i]: c64 [C_i][P_i][R_i]; outs[i]: float [S_i][K_i][R_i]; both arrays
 * are HOST arrays of n_cpi device pointers.
 *
 * With n_cpi == 1 and a tuned slab count above 1 (stap_plan_autotune or
 * stap_plan_set_tuning), the range axis is cut into that many slabs of whole
 * training blocks and each slab's chain runs on its own internal stream,
 * earlier slabs at higher priority, so that the FP64 solve of one slab
 * overlaps the other steps of the next; the result is the same.  Those
 * streams are created by the first such call and joined back into the plan's
 * stream before the call returns.
 *
 * With n_cpi > 1 the CPIs are packed, in order, into waves whose
 * intermediates fit in the workspace beyond step_bytes (any workspace of at
 * least run_bytes works; stap_plan_batch_bytes gives the size at which all
 * CPIs run in one wave).  Within a wave the CPIs run by the plan's batch
 * schedule (stap_plan_set_batch_schedule): phase by phase in persistent
 * launches over all the wave's CPIs (the default), or each CPI's chain on
 * one of several internal streams.  The launch sequence is captured into a
 * CUDA graph on the first call and replayed by later calls that pass the
 * same cubes, outs, workspace and stream; any change re-captures it.  The
 * first batched call also creates the plan's internal streams and events,
 * and (persistent schedule) uploads the per-CPI parameter blocks to the
 * workspace synchronously, before the capture. */
stap_status stap_run_cpi(stap_plan plan, const void* const* cubes, float* const* outs);

/* How stap_run_cpi schedules a batch (n_cpi > 1) within each wave:
 *   STAP_BATCH_PERSISTENT  phase by phase (Doppler, covariance, training,
 *                          solve, apply): the launches that the CPIs of the
 *                          wave need are grouped by kernel, and each group
 *                          runs as ONE persistent launch whose CTAs pull the
 *                          next work item (a CPI's block of range cells,
 *                          bins or systems) from an atomic counter over a
 *                          device array of per-CPI parameter blocks, with no
 *                          waits between CTAs; kernels without a persistent
 *                          form (the mixed-precision refinement solves, the
 *                          training averages, the tensor-core kernels) run
 *                          one launch per CPI in that phase.  The default.
 *   STAP_BATCH_STREAMS     each CPI's four-step chain on one of several
 *                          internal streams, so that CPIs overlap.
 * Either way the whole sequence is captured into a CUDA graph and replayed
 * (see stap_run_cpi).  The results are the same.  stap_plan_autotune times
 * both for a batch plan and keeps the faster. */
typedef enum { STAP_BATCH_PERSISTENT = 0, STAP_BATCH_STREAMS = 1 } stap_batch_schedule;
stap_status stap_plan_set_batch_schedule(stap_plan plan, int32_t schedule);
stap_status stap_plan_get_batch_schedule(stap_plan plan, int32_t* schedule);

/* Workspace size at which every CPI of the plan has its own intermediates,
 * i.e. stap_run_cpi runs the whole batch as one wave. */
stap_status stap_plan_batch_bytes(stap_plan plan, size_t* all_concurrent_bytes);

/* Reduced-DOF front end (not in the paper, whose cubes have 1000 channels,
 * i.e. D = 1000 T): the n_elem element channels of an element cube
 * x[N][P][R] (a half-wavelength line array, element n answering a plane wave
 * of spatial frequency f with exp(j 2 pi f n)) are combined into the plan's C
 * channels by the matrix W[C][N] (host c128, row-major, copied):
 *   cube[c][p][r] = sum_{n<N} conj(W[c][n]) x[n][p][r]
 * (e.g. W[c][n] = 1 on C contiguous subarrays of N/C elements).  The plan's
 * default steering becomes the reduced one,
 *   v_s[t*C + c] = g_t b_s[c],  b_s[c] = sum_n conj(W[c][n]) exp(j 2 pi f_s n),
 * which is the snapshot of a unit plane-wave target, and stays separable.
 * Single-CPI plans only; call once, before stap_plan_set_workspace: it adds W
 * to the run workspace and the element chunk buffers to the stream
 * workspace (stap_plan_workspace_sizes, stap_plan_stream_bytes).  The
 * reduction goes chunk_elems elements at a time (< 1: about 512 MB of element
 * rows), each chunk summed in FP32 and added to the running result.  With a
 * front end, stap_run_stream takes HOST element cubes c64 [N][P][R] and copies
 * them in chunk by chunk. */
stap_status stap_plan_set_front_end(stap_plan plan, int32_t n_elem, const double* W_c128,
                                    int32_t chunk_elems);

/* The front end on the device: elem_cube c64 [N][P][R] -> cube c64 [C][P][R],
 * in one pass over all N elements (the same bits as a streamed run whose
 * chunk holds all N elements).  STAP_ERR_INVALID_ARG if the plan has no front
 * end. */
stap_status stap_reduce_channels(stap_plan plan, const void* elem_cube_c64, void* cube_c64);

/* Workspace size stap_run_stream needs: run_bytes plus two device cubes and
 * two device outputs.  Single-CPI plans only (STAP_ERR_INVALID_ARG
 * otherwise).  Host-only. */
stap_status stap_plan_stream_bytes(stap_plan plan, size_t* bytes);

/* Stream n CPIs of a single-CPI plan's shape from host memory through the
 * whole chain (a runtime feature with no counterpart in the paper, whose GPU
 * tasks copy each cube in and each result back in turn): for i = 0 .. n-1,
 * host_cubes[i] (HOST c64 [C][P][R]) is copied to one of two device cube
 * buffers, stap_run_cpi's chain runs on it, and its output is copied to
 * host_outs[i] (HOST float [S][K][R]).  The copies run on two internal
 * streams, so that the copy-in of CPI i+1 and the copy-out of CPI i-1
 * overlap the chain of CPI i; with page-locked host buffers (cudaHostAlloc,
 * torch pin_memory) a long stream then runs at the rate of the slowest of the
 * three.  Pageable buffers also work, with less overlap.
 *
 * host_cubes, host_outs: HOST arrays of n host pointers; every buffer must
 * stay valid, and the cubes unmodified, until the plan's stream has passed
 * the call: the plan's stream waits for the last copy-out, so synchronising it
 * makes every host_outs[i] ready.  Needs a workspace of at least
 * stap_plan_stream_bytes (else STAP_ERR_NO_WORKSPACE).  n == 0 queues nothing.
 * Returns once everything is queued.  The first call creates the two copy
 * streams and their events. */
stap_status stap_run_stream(stap_plan plan, int64_t n, const void* const* host_cubes,
                            float* const* host_outs);

/* Size of the device scratch array that libstap itself holds for
 * stap_run_cpi_noalloc: 16 MiB on every GPU that loads the library, kept
 * until the process exits. */
#define STAP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* No-allocation form of stap_run_cpi for one CPI.  The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * themselves -- for example a real-time radar loop that forbids cudaMalloc
 * after start-up (it can synchronise the whole device and its latency is
 * unbounded), or a host application whose own pool owns all device memory and
 * gives none to libraries.  Such callers cannot provide the workspace that
 * stap_run_cpi needs, so this call uses a fixed scratch array inside the
 * library (STAP_NOALLOC_SCRATCH_BYTES) instead, and makes no cudaMalloc,
 * cudaFree or other allocating call.
 *
 * dims/opt (opt may be NULL) describe the CPI as for stap_plan_create;
 * cube_c64: device c64 [C][P][R]; out: device float [S][K][R]; cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  If n_failed_systems is not
 * NULL the call waits for the stream and stores the number of covariances
 * that were not positive definite (returning STAP_ERR_NOT_POSDEF if > 0);
 * otherwise it returns as soon as the work is queued.
 *
 * Errors: the shape/option errors of stap_plan_create; STAP_ERR_NO_WORKSPACE
 * if the CPI needs more scratch than STAP_NOALLOC_SCRATCH_BYTES (the
 * stap_plan_workspace_sizes run_bytes of the same dims), rejected before any
 * CUDA call; STAP_ERR_CUDA if a CUDA call fails.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and keeps it; make that first call before any stream
 * capture begins.  Every call on a device shares the one array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and give
 * wrong results, so order them.  Each call clears the status it uses and
 * rewrites the tables and intermediates before reading them. */
stap_status stap_run_cpi_noalloc(const stap_dims* dims, const stap_options* opt, void* cuda_stream,
                                 const void* cube_c64, float* out, int64_t* n_failed_systems);

/* Number of launch choices per CPI kept by the autotuner. */
#define STAP_TUNING_LEN 9

/* Autotune the launch configuration of every distinct CPI shape of the plan
 * (C, P, K, T, B, S; CPIs that differ only in R share one tuning): for each
 * step in turn it times candidate tile shapes and schedules on the device, on
 * the caller's cubes and output buffers, `reps` runs each (reps < 1 means 3),
 * and keeps the fastest.  Candidates: range cells per Doppler CTA (8/16/32);
 * Doppler bins per covariance CTA (plain precision); lanes per system and
 * warps per CTA of the D <= 32 solve, lanes per right-hand side of the larger
 * solve, and for D = 8, 12 or 16 the register-resident or the shared-memory
 * solve kernel; register-resident or general FP32 apply; for a one-CPI plan, 1, 2, 3,
 * 4, 6 or 8 pipelined range slabs of the whole run; for the mixed precisions
 * (STAP_PREC_BF16X3, STAP_PREC_TF32X3, STAP_PREC_FP16_SCALED), the tensor-core
 * or the FP32 covariance and apply (the FP32 kernels are the more accurate,
 * and at small D the faster); for a batch, the persistent or the stream
 * schedule (stap_plan_set_batch_schedule).  Every candidate computes
 * the same result except that the apply kernels sum in different orders and
 * that a mixed-precision plan's FP32 choices are more accurate than its
 * tensor-core ones.  Needs the run workspace; synchronises the plan's stream; overwrites
 * outs; clears the device status; drops a captured batch graph. */
stap_status stap_plan_autotune(stap_plan plan, const void* const* cubes, float* const* outs,
                               int32_t reps);

/* The launch choices of CPI `cpi` as STAP_TUNING_LEN integers (0 = built-in
 * heuristic): Doppler cells per CTA, covariance bins per CTA, solve lanes per
 * system, solve warps per CTA, large-solve lanes per right-hand side, apply
 * kernel (1 register-resident, 2 general), range slabs of a one-CPI
 * stap_run_cpi (at most 8 and NB are used), solve kernel for D <= 32
 * (1 register-resident for D = 8, 12, 16, 2 shared-memory teams, 3 one
 * system per CTA), covariance of a mixed-precision
 * plan (1 FP32, 2 tensor cores; apply choice 3 = tensor cores).  set_tuning installs saved choices
 * (values 0..64; a choice that does not fit a launch falls back to the
 * heuristic). */
stap_status stap_plan_get_tuning(stap_plan plan, int32_t cpi, int32_t* choices);
stap_status stap_plan_set_tuning(stap_plan plan, int32_t cpi, const int32_t* choices);

/* Wait for the plan's stream, then report and clear the device status.
 * *n_failed_systems (if not NULL) = covariances found not positive definite
 * since the last call; returns STAP_ERR_NOT_POSDEF if that is > 0,
 * STAP_ERR_TIMEOUT if a bounded device wait gave up, else STAP_OK. */
stap_status stap_get_status(stap_plan plan, int64_t* n_failed_systems);

/* Static description of a status code. */
const char* stap_status_string(stap_status status);

/* Test support: out[i] = the reciprocal 1/in[i] exactly as the FP64
 * factorisation of the one-system-per-CTA solve forms its pivots' reciprocals
 * (Newton-Raphson iteration from the hardware's approximate reciprocal), so
 * that a test can compare it with IEEE division.  in, out: n device doubles
 * (in[i] positive, finite and normal; other values give unspecified results);
 * runs on cuda_stream (NULL = legacy default stream) and waits for it.
 * Errors: STAP_ERR_INVALID_ARG for n < 0 or NULL pointers with n > 0;
 * STAP_ERR_CUDA.  No counterpart in the paper. */
stap_status stap_test_pivot_reciprocal(const double* in, double* out, int64_t n, void* cuda_stream);

/* 1 if this library is the checked build (compiled with -DSTAP_CHECKED),
 * else 0.  No counterpart in the paper: a debugging aid. */
int32_t stap_checked_build(void);

/* Checked build only: every kernel compares each index into a global buffer
 * (and the tensor-core kernels each shared- and tensor-memory offset) with
 * the extent of that buffer as the launch sees it, skips an access outside
 * it and records it; nothing traps.  This call waits for the current device,
 * then reports and clears the records of all kernels on it: *count = accesses
 * skipped since the last call; *site (a code naming the kind of access: 1/2
 * Doppler input/output, 3/4 covariance input/output, 5/6 solve input/output,
 * 7/8 apply input/output, 9/10 tensor-core input/output, 11 tensor-core
 * shared memory, 12 tensor memory, 13 training matrices), *index and *extent
 * of the first one found (site, index, extent may be NULL).  The normal build
 * returns STAP_ERR_UNSUPPORTED with *count = 0.  No counterpart in the paper:
 * a debugging aid. */
stap_status stap_check_report(int64_t* count, int32_t* site, int64_t* index, int64_t* extent);

/* STAP_ABI_VERSION of the loaded library. */
int32_t stap_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STAP_H_ */
