"""Benchmark of the STAP path on GB300: range-Doppler cells per second.

One step = one whole CPI through ``stap_run_cpi`` (Doppler transform,
covariance, FP64 loading/LDL^H/solves/refinement, apply).  The headline is the
large CPI (C=32 channels, P=512 pulses, K=512 Doppler bins, R=32768 range
cells, T=4 so D=128, B=256-cell training blocks, S=64 steering vectors; a
seeded synthetic 4.3 GB cube: unit noise, 40 dB CNR clutter ridge, 32
targets) on the mixed path (FP16 per-block-scaled split products on the tensor
cores for the covariance and the apply, FP64 solve), with the plain FP32 path
timed on the same cube beside it.  The D = 64 CPI, the standard D = 12 CPI and
the 512-CPI batch are keys of the same line, each with its mixed and plain
legs; every single-CPI workload also runs the mixed-precision refinement
solve, and the standard CPI runs the training and snapshot options.  Errors
against the FP64 oracle on seeded range blocks accompany every leg.

Timing: inputs resident in HBM, L2 flushed (256 MiB write) between timed steps,
each step bracketed by CUDA events on the launching stream; barrier and
synchronize around the timed region; max over ranks.  Under torchrun every rank
processes its own CPIs (weak scaling, no data-path collective).

``--impl reference`` times the FP64 CPU oracle on the host cores instead (rank
0 only), each step a bounded sample of the same workload.
"""
import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "STAP range-Doppler cells/s per GB300, mixed vs FP32 at ≤1e-3 err vs FP64"
UNIT = "cells/s"
NAME = "large"
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) per launch of the solve kernel (dram__bytes_read.sum
# + dram__bytes_write.sum of one unslabbed launch, from an ncu capture
# summarised in profiles/), keyed by a hash of the kernel source, the solve
# kernel the tuning chose (1 register-resident, 2 shared-memory teams, 3 one
# system per CTA) and the workload, so that a changed or different kernel
# reports null until re-measured.  The large CPI's entry is an eighth of it
# (8192 of its 65536 systems, same kernel and launch shape: 1151412224 bytes
# read + 510120448 written, the capture summarised in profiles/) scaled by 8, the
# traffic being per system (its lower triangle read, its weights written).
# The second key is solve.cu after a change confined to the refinement
# option's team kernel (solve_mir_kernel, its shared-memory strides and size
# function, and a helper they use): solve_big_kernel's source is the same, so
# the same capture applies.
SOLVE_TRAFFIC = {("ece189e7f5967c5d", 3, "large"): 8 * (1151412224 + 510120448),
                 ("077ece954fb9fac1", 3, "large"): 8 * (1151412224 + 510120448)}
SOLVE_KERNELS = {1: "solve_reg_kernel (register-resident FP64 LDL^H, solves, refinement)",
                 2: "solve_kernel (shared-memory FP64 Cholesky teams, solves, refinement)",
                 3: "solve_big_kernel (one system per CTA: FP64 LDL^H, solves, refinement)"}


def peaks():
    """Roofline denominators: MEASURED_PEAKS.json (HBM copy bandwidth, cuBLAS
    bf16 burst and sustained) when present, else the recipe's fallbacks; FP64
    and FP32 ALU peaks from unit counts and the maximum SM clock."""
    p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "bf16_tflops": float(m.get("bf16_tflops", 1900.0)),
             "bf16_tflops_sustained": float(m.get("bf16_tflops_sustained", 1700.0)), "src": "measured"}
    # FP64 / FP32 ALU peaks from unit counts and the maximum SM clock:
    # 152 SMs x 2 DFMA lanes/clk (x2 flops) and x 128 FFMA lanes/clk (x2 flops) at 2070 MHz.
    p["fp64_tflops"] = 152 * 2 * 2 * 2.070e9 / 1e12
    p["fp32_tflops"] = 152 * 128 * 2 * 2.070e9 / 1e12
    return p


def workload_spec(rank=0, name="standard"):
    import dataclasses
    from paper_2203_06233_gb300 import synth
    return dataclasses.replace(synth.WORKLOADS[name](), sub=rank)


def workload_config(spec, name=None):
    C, P, K, R, T, B, S = spec.dims()
    name = name or NAME
    return {"workload": f"{name} CPI C{C} P{P} K{K} R{R} T{T} B{B} S{S} (D={C*T}), "
                        f"{spec.cnr_db:.0f} dB CNR, {len(spec.targets)} targets",
            "n_chan": C, "n_pulses": P, "n_dop": K, "n_range": R, "tdof": T,
            "training_block": B, "n_steering": S, "cells_per_step": K * R,
            "l2": "flushed between timed steps (256 MiB write); inputs resident in HBM",
            "parallelism": "one CPI per GPU per step"}


def solve_flops(spec, refine=1, separable=True):
    """Algorithmic FP64 flops of the loading/Cholesky/solve kernel (8 flops per
    complex multiply-add): Cholesky D^3/6, then (1 + 2 refine) forward/back
    solve pairs of D^2 each (one solve, then per refinement step a residual
    and a solve) for each right-hand side -- the C basis vectors when the
    steering set is separable, otherwise the S steering vectors, followed by
    their FP64 normalisations (D real products each).  The separable path's
    combination of the basis solutions and its normalisations run in
    double-float on the FP32 pipe and are not FP64 work."""
    C, P, K, R, T, B, S = spec.dims()
    D, NB = C * T, R // B
    if separable:
        per = 8.0 * (D ** 3 / 6.0 + (1 + 2 * refine) * C * D * D)
    else:
        per = 8.0 * (D ** 3 / 6.0 + (1 + 2 * refine) * S * D * D) + 4.0 * S * D
    return K * NB * per


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        # the raw samples go to $STAP_CLOCK_LOG_DIR (kept) or the temporary directory
        d = os.environ.get("STAP_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"stap_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[3][1:]) if v.lower() == "active"})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def aggregate(local_ms, local_cells, world, device):
    """Whole-job throughput: every rank processed ``local_cells`` (weak scaling)
    in ``local_ms``; the job took the slowest rank's time.  Returns
    (max time over ranks in ms, all ranks' cells per second)."""
    import torch
    total_ms = float(local_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * local_cells / (total_ms * 1e-3)


def slab_count(tuning, nb):
    """Range slabs the tuned one-CPI run uses (four kernel launches each)."""
    (choices,) = tuning.values()
    return max(1, min(choices[6], 8, nb))


def time_steps(fn, steps, flush, stream):
    """Per-step device time (ms) with CUDA events, L2 flushed before each step."""
    import torch
    evs = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def power_errors(got, ref):
    """Normwise relative error of the output power, and the worst cell
    relative to its own power floored at the median power."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    normwise = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    floor = np.maximum(ref, np.median(ref))
    return {"normwise": normwise, "max_cell": float(np.max(np.abs(got - ref) / floor))}


# mixed-precision arithmetic of each workload's mixed leg (the configurations'
# stated precision: FP16 with per-block scaling for the large CPI, BF16 split
# products for the D = 64 CPI and the batch; the D = 12 CPIs have no stated
# mixed arithmetic and take BF16X3 as the more accurate split)
MIXED_PREC = {"large": ("fp16_scaled", 3), "mixed": ("bf16x3", 1), "mixed_small": ("bf16x3", 1),
              "standard": ("bf16x3", 1), "small": ("bf16x3", 1), "batch": ("bf16x3", 1)}
PREC_NAMES = {0: "fp32", 1: "bf16x3", 2: "tf32x3", 3: "fp16_scaled"}
PREC_TEXT = {
    0: "plain: FP32 FFT, covariance accumulated error-free in FP32 pairs, FP32 apply",
    1: "mixed: BF16 three-piece split products (6) on the tensor cores for covariance and apply, "
       "FP32 accumulation; FP32 FFT",
    2: "mixed: TF32 two-piece split products (3) on the tensor cores for covariance and apply, "
       "FP32 accumulation; FP32 FFT",
    3: "mixed: FP16 two-piece split products (3) with per-block power-of-two scaling on the tensor "
       "cores for covariance and apply, FP32 accumulation; FP32 FFT",
}
SOLVE_TEXT = "FP64 diagonal load, LDL^H factorisation and substitutions, 1 refinement step"
MIR_TEXT = ("mixed-precision refinement solve: FP64 diagonal load, FP32 LDL^H and substitutions, "
            "2 refinement steps with double-float residuals (STAP_SOLVE_MIXED_IR)")


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def sample_blocks(spec, n):
    """n seeded range blocks of the CPI (all of them if it has fewer)."""
    rng = np.random.default_rng(1234 + spec.seed)
    n = min(n, spec.NB)
    return sorted(int(b) for b in rng.choice(spec.NB, n, replace=False))


def oracle_on_blocks(spec, cube_h, blocks):
    """The FP64 oracle, as it stands, on each sampled block's range window
    (blocks are independent: the Doppler transform is per range cell, the
    snapshots and training stay inside the block).  Returns ({block: output
    [S][K][B]}, the cpu_baseline dict)."""
    import oracle
    d = oracle.Dims(*spec.dims())
    B = spec.training_block
    refs = {}
    t0 = time.perf_counter()
    for b in blocks:
        refs[b] = oracle.run(d, cube_h, r0=b * B, nr=B)["out"]
    el = time.perf_counter() - t0
    cells = len(blocks) * B * spec.n_dop
    base = {"value": cells / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(blocks)} seeded range block(s) of {B} cells x {spec.n_dop} bins of "
                      f"the {NAME_OF.get(spec.dims(), 'CPI')} CPI, all eight steps on each window, "
                      f"{cells} cells in {el:.1f} s"}
    return refs, base


NAME_OF = {}


def block_errors(outs_blocks, refs):
    """Errors of one leg over the sampled blocks: normwise over all of them
    and the worst cell (relative to max(P, median P) of its block)."""
    num = den = 0.0
    worst = 0.0
    for b, ref in refs.items():
        got = outs_blocks[b].astype(np.float64)
        num += float(np.sum((got - ref) ** 2))
        den += float(np.sum(ref ** 2))
        worst = max(worst, power_errors(got, ref)["max_cell"])
    return {"normwise": (num / den) ** 0.5, "max_cell": worst, "blocks": len(refs)}


def kernel_figures(spec, prec, kt, pk, refine=1, solver=0, used=None):
    """Each step against its own bound: achieved rate and fraction.  `used`
    (the leg's kernels_used) says which kernel ran the covariance and the
    apply: a mixed plan keeps the FP32 kernel of a step where the autotuner
    found it faster."""
    if not kt:
        return {}
    C, P, K, R, T, B, S = spec.dims()
    D, NB = C * T, R // B
    dop_bytes = 8.0 * C * R * (P + K)
    sf = solve_flops(spec, refine=refine)
    out = {
        "doppler": {"ms": kt["doppler"], "bound": "hbm", "bytes": dop_bytes,
                    "achieved_gbs": dop_bytes / kt["doppler"] / 1e6,
                    "frac": dop_bytes / kt["doppler"] / 1e6 / pk["hbm_gbs"]},
        "solve": {"ms": kt["solve"], "bound": "alu", "fp64_flops": sf,
                  "achieved_tflops": sf / kt["solve"] / 1e9,
                  "frac": sf / kt["solve"] / 1e9 / pk["fp64_tflops"]},
    }
    if solver == 1:   # FP32 factor and substitutions, double-float residuals: no FP64 roofline
        out["solve"] = {"ms": kt["solve"], "bound": "fp32 issue",
                        "fp64_equivalent_tflops": sf / kt["solve"] / 1e9,
                        "note": "FP64-solve flop count over this solve's time, for comparison with "
                                "the FP64 solve; the kernel itself runs on the FP32 and integer pipes"}
    # covariance through the step call (full Hermitian c128 output)
    cov_bytes = 8.0 * C * K * R + 16.0 * K * NB * D * D
    apply_bytes = 8.0 * C * K * R + 8.0 * K * NB * S * D + 4.0 * S * K * R
    used = used or {}
    fp32_cov = prec == 0 or used.get("covariance", "").startswith("FP32")
    fp32_app = prec == 0 or used.get("apply", "").startswith("FP32")
    if fp32_cov:
        cplx = 1.0 * K * NB * B * (T * C * C - C * (C - 1) // 2)
        out["covariance"] = {"ms": kt["covariance"], "bound": "alu", "fp32_instr": 20.0 * cplx,
                             "frac": 20.0 * cplx / kt["covariance"] / 1e9 / (pk["fp32_tflops"] / 2),
                             "hbm_frac": cov_bytes / kt["covariance"] / 1e6 / pk["hbm_gbs"]}
    if fp32_app:
        af = 8.0 * K * R * S * D
        out["apply"] = {"ms": kt["apply"], "bound": "alu", "fp32_flops": af,
                        "frac": af / kt["apply"] / 1e9 / pk["fp32_tflops"],
                        "hbm_frac": apply_bytes / kt["apply"] / 1e6 / pk["hbm_gbs"]}
    if prec != 0:
        nprod = 6 if prec == 1 else 3
        peak = pk["bf16_tflops"] / (2.0 if prec == 2 else 1.0)
        # tensor work the kernels issue (real MACs), D8 = D rounded up to 8 and
        # NA = G D8 rounded up to 16:
        #   covariance, D8 <= 64 (stacked [Xr ; Xi] rows, G = 64 // D8 systems
        #   per tile): 2 MMAs of 128 x NA per K step; D8 > 64 (G = 1): 4 of
        #   128 x NA; K = B cells, nprod products;
        #   apply: 128 x NP x 2D per 128-cell tile (NP = 2 S per block in the
        #   tile, rounded up to 16)
        D8 = (D + 7) // 8 * 8
        G, nmma = (64 // D8, 2) if D8 <= 64 else (1, 4)
        NA = -(-G * D8 // 16) * 16
        cov_mac = nmma * 128.0 * NA * B * np.ceil(K * NB / G) * nprod
        nbt = 128 // B if B < 128 else 1
        NP = -(-2 * nbt * S // 16) * 16
        app_mac = 128.0 * NP * 2 * D * K * np.ceil(R / 128) * nprod
        # useful work: the four real blocks of each system's own D x D
        # covariance (the Hermitian half is not exploited), the apply's
        # 4 real products per complex one
        cov_useful = 2.0 * 4 * D * D * B * K * NB * nprod
        for name, mac, useful, byts, skip in (
                ("covariance", cov_mac, cov_useful, cov_bytes, fp32_cov),
                ("apply", app_mac, 2.0 * 4 * D * S * K * R * nprod, apply_bytes, fp32_app)):
            if skip:
                continue
            out[name] = {"ms": kt[name], "bound": "tensor", "issued_tflops": 2 * mac / kt[name] / 1e9,
                         "useful_tflops": useful / kt[name] / 1e9,
                         "frac": 2 * mac / kt[name] / 1e9 / peak,
                         "hbm_gbs": byts / kt[name] / 1e6,
                         "hbm_frac": byts / kt[name] / 1e6 / pk["hbm_gbs"],
                         "peak_tflops": peak}
    return out


def run_leg(spec, cube, dev, prec, args, flush, stream, kernel_reps, timed=None, barrier=None,
            solver=0, refine=1, opts=None, label=None):
    """One path on the workload's cube: plan (with the plan options `opts`),
    autotune (untimed), warm-up, args.steps timed steps (after `barrier()` and
    inside `timed`, a context manager, if given), per-step kernel times;
    returns (plan, out, leg dict)."""
    import contextlib
    import torch
    from paper_2203_06233_gb300 import stap
    C, P, K, R, T, B, S = spec.dims()
    plan = stap.Plan(spec.dims(), device=dev, precision=prec, solver=solver, refine_steps=refine,
                     **(opts or {}))
    out = torch.empty((S, K, R), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    tuning = plan.autotune(cube, out, reps=1 if K * R * C * T > (1 << 26) else 3)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        flush()
        plan.run_cpi(cube, out)
    torch.cuda.synchronize()
    code, failed = plan.status()
    if code != stap.STAP_OK:
        raise RuntimeError(f"{PREC_NAMES[prec]}: device status {code} ({failed} failed systems)")
    if barrier is not None:
        barrier()
    with (timed if timed is not None else contextlib.nullcontext()):
        # the headline's timed steps are bracketed for a profiler started with
        # profiling off (ncu --profile-from-start off sees exactly their launches)
        if timed is not None:
            torch.cuda.profiler.start()
        times = time_steps(lambda: plan.run_cpi(cube, out), args.steps, flush, stream)
        if timed is not None:
            torch.cuda.profiler.stop()
    plan.run_cpi(cube, out)
    torch.cuda.synchronize()
    code, failed = plan.status()
    if code != stap.STAP_OK:
        raise RuntimeError(f"{PREC_NAMES[prec]}: device status {code} ({failed} failed systems)")
    # per-kernel times through the step-by-step calls (same launch choices)
    kt = {}
    if not opts:   # the training options add a step between covariance and solve
        dop = plan.doppler(cube)
        cov = plan.covariance(dop)
        wts = plan.solve_weights(cov)
        kt = {
            "doppler": statistics.mean(time_steps(lambda: plan.doppler(cube, dop), kernel_reps, flush, stream)),
            "covariance": statistics.mean(time_steps(lambda: plan.covariance(dop, cov), kernel_reps, flush,
                                                     stream)),
            "solve": statistics.mean(time_steps(lambda: plan.solve_weights(cov, wts), kernel_reps, flush,
                                                stream)),
            "apply": statistics.mean(time_steps(lambda: plan.apply(dop, wts, out), kernel_reps, flush, stream)),
        }
        plan.run_cpi(cube, out)   # the run's own output again (the apply call above rewrote it)
        del dop, cov, wts
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    (choices,) = tuning.values()
    log(f"{spec.dims()} {label or PREC_NAMES[prec]}: {sum(times) / args.steps:.3f} ms/step, "
        f"autotune {tune_s:.1f} s, kernels {kt}")
    leg = {"precision": PREC_NAMES[prec],
           "arithmetic": PREC_TEXT[prec] + "; " + (MIR_TEXT if solver == 1 else SOLVE_TEXT),
           "ms_per_step": sum(times) / args.steps, "step_ms": times, "tuning": tuning,
           "autotune_s": tune_s, "kernels_ms": kt,
           "kernels_used": {"covariance": "FP32 error-free" if prec == 0 or choices[8] == 1 else "tensor cores",
                            "apply": "FP32" if prec == 0 or choices[5] in (1, 2) else "tensor cores"}}
    return plan, out, leg


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2203_06233_gb300 import stap, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flushbuf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def flush():
        flushbuf.zero_()

    pk = peaks()
    line = None
    extra = {}
    # the workload of the headline first, then the other single-CPI workloads
    # as keys of the same line (rank 0 of a one-GPU run only)
    names = [NAME] + ([n for n in ("mixed", "standard") if n != NAME]
                      if world == 1 and not args.only_headline else [])
    for wi, name in enumerate(names):
        head = wi == 0
        if not head:
            try:
                extra[name] = workload_keys(args, name, rank, dev, stream, flush, pk)
            except Exception as exc:   # an extra key must not lose the headline line
                log(f"{name}: {type(exc).__name__}: {exc}")
                extra[name] = {"error": f"{type(exc).__name__}: {exc}"[:400]}
            torch.cuda.empty_cache()
            continue
        spec = workload_spec(rank, name)
        NAME_OF[spec.dims()] = name
        C, P, K, R, T, B, S = spec.dims()
        cells = K * R
        mname, mprec = MIXED_PREC[name]
        cube = synth.make_cube_torch(spec, dev)
        cube_h = cube.cpu().numpy()
        big = cube_h.nbytes > (1 << 30)
        kernel_reps = 3 if big else max(20, min(200, args.steps))
        blocks = sample_blocks(spec, 8 if name == "large" else 4)
        sub = argparse.Namespace(steps=args.steps if head else max(3, min(args.steps, 10)),
                                 warmup=args.warmup)
        legs, outs_blocks = {}, {}
        clk = ClockSampler(local) if head else None
        mplan = mout = None

        def barrier():
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()

        mlabel, flabel, ilabel = PREC_NAMES[mprec], PREC_NAMES[0], PREC_NAMES[mprec] + "+mixed_ir"
        short = argparse.Namespace(steps=max(3, min(args.steps, 5)), warmup=args.warmup)
        for label, prec, solver, refine in ((mlabel, mprec, 0, 1), (flabel, 0, 0, 1), (ilabel, mprec, 1, 2)):
            keep = head and label == mlabel        # the headline leg: timed with clocks, kept for e2e
            if label == ilabel and (world > 1 or args.only_headline):
                continue
            try:
                plan, out, leg = run_leg(spec, cube, dev, prec, sub if label != ilabel else short, flush,
                                         stream, kernel_reps, timed=clk if keep else None,
                                         barrier=barrier if keep else None, solver=solver, refine=refine,
                                         label=label)
            except Exception as exc:
                if label != ilabel:
                    raise
                log(f"{label}: {type(exc).__name__}: {exc}")   # a side leg must not lose the line
                torch.cuda.empty_cache()
                continue
            outs_blocks[label] = {b: out[:, :, b * B:(b + 1) * B].cpu().numpy() for b in blocks}
            legs[label] = leg
            if keep:
                mplan, mout = plan, out
            else:
                plan.close()
                del plan, out
                torch.cuda.empty_cache()
        mleg, fleg = legs[mlabel], legs[flabel]
        errors, cpu = {}, None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            refs, cpu = oracle_on_blocks(spec, cube_h, blocks)
            errors = {lb: block_errors(outs_blocks[lb], refs) for lb in outs_blocks}
        mvalue = world * cells / (mleg["ms_per_step"] * 1e-3)
        fvalue = world * cells / (fleg["ms_per_step"] * 1e-3)
        # ---- headline: the mixed leg's timed region ----
        total_ms, value = aggregate(mleg["ms_per_step"] * sub.steps, cells * sub.steps, world, dev)
        ms_per_step = total_ms / sub.steps
        kern = kernel_figures(spec, mprec, mleg["kernels_ms"], pk, used=mleg["kernels_used"])
        solve_kind = 3 if C * T > 32 else list(mleg["tuning"].values())[0][7]
        roofline = {"kernel": SOLVE_KERNELS.get(solve_kind, "solve"),
                    "bound": "alu", "achieved": kern["solve"]["achieved_tflops"],
                    "peak": pk["fp64_tflops"], "unit": "TFLOP/s", "frac": kern["solve"]["frac"],
                    "traffic": SOLVE_TRAFFIC.get((kernel_hash(), solve_kind, name)),
                    "basis": "8 K NB (D^3/6 + (1 + 2 refine) C D^2) FP64 flops per launch: the "
                             "factorisation plus, for each of the C basis right-hand sides of the "
                             "separable steering (v_s = g (x) a_s), one forward/back solve pair and "
                             "per refinement step a residual and a solve pair; the combination into "
                             "the S steering vectors and their normalisation run on the FP32 pipe",
                    "peak_src": "FP64: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (unit count and max "
                                "clock; a DFMA microbenchmark measured 1.20 TFLOP/s at 1987 MHz)"}
        # ---- end to end through the public API from pinned host buffers ----
        ring = 4 if cube_h.nbytes <= (1 << 30) else 2
        cube_pin = torch.from_numpy(cube_h).pin_memory()
        host_cubes = [cube_pin] + [cube_pin.clone().pin_memory() for _ in range(ring - 1)]
        host_outs = [torch.empty((S, K, R), dtype=torch.float32).pin_memory() for _ in range(ring)]
        n_stream = max(2 * ring, min(sub.steps, 10 if big else 1000))
        mplan.run_stream(host_cubes[:2], host_outs[:2])      # warm-up (grows the workspace once)
        torch.cuda.synchronize()
        seq_c = [host_cubes[i % ring] for i in range(n_stream)]
        seq_o = [host_outs[i % ring] for i in range(n_stream)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mplan.run_stream(seq_c, seq_o)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms, _ = aggregate(e0.elapsed_time(e1), cells * n_stream, world, dev)
        e2e_ms /= n_stream
        code, failed = mplan.status()
        if code != stap.STAP_OK:
            raise RuntimeError(f"e2e: device status {code} ({failed} failed systems)")
        del host_cubes, host_outs, cube_pin, seq_c, seq_o
        cfg = workload_config(spec, name)
        cfg["precision"] = mleg["arithmetic"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": sub.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[mprec], "data": "synthetic",
            "config": cfg,
            "e2e": {"value": world * cells / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": cube_h.nbytes, "d2h_bytes_per_step": S * K * R * 4,
                    "ms_per_step": e2e_ms,
                    "api": f"stap_run_stream over {n_stream} CPIs from a ring of {ring} pinned host "
                           "cubes and outputs: every CPI copied in, run and copied out inside the "
                           "timed region, copies overlapping the neighbouring CPIs' chains"},
            "gpu_launches": 4 * slab_count(mleg["tuning"], R // B) * sub.steps,
            "mixed": dict(mleg, value=value, kernels=kern),
            "fp32": dict(fleg, value=world * cells / (fleg["ms_per_step"] * 1e-3),
                         kernels=kernel_figures(spec, 0, fleg["kernels_ms"], pk)),
            "mixed_vs_fp32": value / (world * cells / (fleg["ms_per_step"] * 1e-3)),
            "roofline": roofline,
            "clocks": clk.summary(),
        }
        if ilabel in legs:
            ileg = legs[ilabel]
            line["mixed_ir"] = dict(ileg, value=world * cells / (ileg["ms_per_step"] * 1e-3),
                                    kernels=kernel_figures(spec, mprec, ileg["kernels_ms"], pk, solver=1,
                                                           used=ileg["kernels_used"]))
        if errors:
            line["errors_vs_oracle"] = errors
        if cpu is not None:
            line["cpu_baseline"] = cpu
        mplan.close()
        del mout, cube
        torch.cuda.empty_cache()
    if extra:
        line["workloads"] = extra
    if world == 1 and not args.only_headline and NAME == "large":
        try:
            line["workloads"]["batch"] = batch_legs(args, dev, stream, flush)
        except Exception as exc:   # an extra key must not lose the headline line
            log(f"batch: {type(exc).__name__}: {exc}")
            line["workloads"]["batch"] = {"error": f"{type(exc).__name__}: {exc}"[:400]}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def workload_keys(args, name, rank, dev, stream, flush, pk):
    """Another single-CPI workload as a key of the line: its mixed and FP32
    legs and the mixed leg with the mixed-precision refinement solve (a few
    timed steps each), their errors on sampled blocks, and on the standard CPI
    the option legs."""
    import torch
    from paper_2203_06233_gb300 import synth
    spec = workload_spec(rank, name)
    NAME_OF[spec.dims()] = name
    C, P, K, R, T, B, S = spec.dims()
    cells = K * R
    mprec = MIXED_PREC[name][1]
    cube = synth.make_cube_torch(spec, dev)
    cube_h = cube.cpu().numpy()
    kernel_reps = 3 if cube_h.nbytes > (1 << 30) else max(20, min(200, args.steps))
    blocks = sample_blocks(spec, 4)
    sub = argparse.Namespace(steps=max(3, min(args.steps, 10)), warmup=args.warmup)
    legs, outs_blocks = {}, {}
    mlabel, flabel, ilabel = PREC_NAMES[mprec], PREC_NAMES[0], PREC_NAMES[mprec] + "+mixed_ir"
    for label, prec, solver, refine in ((mlabel, mprec, 0, 1), (flabel, 0, 0, 1), (ilabel, mprec, 1, 2)):
        plan, out, leg = run_leg(spec, cube, dev, prec, sub, flush, stream, kernel_reps, solver=solver,
                                 refine=refine, label=label)
        outs_blocks[label] = {b: out[:, :, b * B:(b + 1) * B].cpu().numpy() for b in blocks}
        legs[label] = leg
        plan.close()
        del plan, out
        torch.cuda.empty_cache()
    errors, cpu = {}, None
    if not args.no_cpu_baseline:
        refs, cpu = oracle_on_blocks(spec, cube_h, blocks)
        errors = {lb: block_errors(outs_blocks[lb], refs) for lb in outs_blocks}
    value = {lb: cells / (legs[lb]["ms_per_step"] * 1e-3) for lb in legs}
    res = {"config": workload_config(spec, name),
           "mixed": dict(legs[mlabel], value=value[mlabel],
                         kernels=kernel_figures(spec, mprec, legs[mlabel]["kernels_ms"], pk,
                                                used=legs[mlabel]["kernels_used"])),
           "fp32": dict(legs[flabel], value=value[flabel],
                        kernels=kernel_figures(spec, 0, legs[flabel]["kernels_ms"], pk)),
           "mixed_ir": dict(legs[ilabel], value=value[ilabel],
                            kernels=kernel_figures(spec, mprec, legs[ilabel]["kernels_ms"], pk, solver=1,
                                                   used=legs[ilabel]["kernels_used"])),
           "mixed_vs_fp32": value[mlabel] / value[flabel], "errors_vs_oracle": errors,
           "cpu_baseline": cpu}
    if name == "standard":
        res["options"] = option_legs(args, spec, cube, cube_h, dev, stream, flush, kernel_reps)
    return res


def option_legs(args, spec, cube, cube_h, dev, stream, flush, kernel_reps):
    """The plain path with each snapshot and training option on the standard
    CPI's cube: PRI-staggered snapshots, neighbour-block training, and a
    sliding training window over groups of 8 cells (1 guard group and 8
    training groups on each side); errors against the oracle run with the same
    option on seeded 64-cell range windows."""
    import torch
    from paper_2203_06233_gb300 import stap
    C, P, K, R, T, B, S = spec.dims()
    cells = K * R
    sub = argparse.Namespace(steps=max(3, min(args.steps, 10)), warmup=args.warmup)
    wspec = dataclasses.replace(spec, training_block=8)
    cases = [
        ("staggered", spec, dict(snapshots=stap.STAP_SNAP_PRI_STAGGERED), dict(staggered=True),
         "PRI-staggered snapshots: T sub-windows of P - T + 1 pulses"),
        ("neighbour_training", spec, dict(training=stap.STAP_TRAIN_NEIGHBOURS), dict(training=1),
         "block b trained on blocks b - 1 and b + 1"),
        ("window_training", wspec, dict(training=stap.STAP_TRAIN_WINDOW, train_guard=1, train_half=8),
         dict(training=2, guard=1, half=8),
         "groups of 8 cells, each trained on 8 groups on each side beyond 1 guard group"),
    ]
    rng = np.random.default_rng(77)
    windows = sorted(int(w) for w in rng.choice(R // 64, 4, replace=False))
    res = {}
    for key, sp, kw, okw, text in cases:
        try:
            plan, out, leg = run_leg(sp, cube, dev, 0, sub, flush, stream, kernel_reps, opts=kw, label=key)
            got = {w: out[:, :, w * 64:(w + 1) * 64].cpu().numpy() for w in windows}
            plan.close()
            del plan, out
            torch.cuda.empty_cache()
            entry = dict(leg, option=text, value=cells / (leg["ms_per_step"] * 1e-3))
            if not args.no_cpu_baseline:
                import oracle
                d = oracle.Dims(*sp.dims())
                refs = {w: oracle.run(d, cube_h, r0=w * 64, nr=64, **okw)["out"] for w in windows}
                entry["errors_vs_oracle"] = block_errors(got, refs)
            res[key] = entry
        except Exception as exc:   # an option leg must not lose the line
            log(f"{key}: {type(exc).__name__}: {exc}")
            res[key] = {"error": f"{type(exc).__name__}: {exc}"[:400]}
    return res


DTYPE = {0: "f32+f64", 1: "bf16x3+f32+f64", 2: "tf32x3+f32+f64", 3: "f16x2+f32+f64"}


def batch_legs(args, dev, stream, flush):
    """The 512-CPI batch (one stap_run_cpi call, a captured graph replayed)
    on the mixed and the plain path, a few steps each; errors on one seeded
    block of 8 seeded CPIs."""
    import torch
    from paper_2203_06233_gb300 import stap, synth
    specs = synth.batch_cpis(512)
    cubes = [synth.make_cube_torch(s, dev) for s in specs]
    cells = sum(s.cells for s in specs)
    rng = np.random.default_rng(4)
    picks = [(i, int(rng.integers(specs[i].NB)))
             for i in sorted(int(x) for x in rng.choice(len(specs), 8, replace=False))]
    res = {"config": {"workload": "batch of 512 uneven CPIs: C in {4,8,16}, T in {2,3,4}, P = K in "
                                  "{64,128,256}, R = 64 x U{16..256}, B 64, S in {8,16}",
                      "cells_per_step": cells, "n_cpi": len(specs)}}
    outs_pick = {}
    steps = max(2, min(args.steps, 3))
    for prec in (MIXED_PREC["batch"][1], 0):
        outs = [torch.empty((s.n_steering, s.n_dop, s.n_range), dtype=torch.float32, device=dev)
                for s in specs]
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        # workspace: as much of the all-concurrent size as free HBM allows (8 GiB spare)
        free = torch.cuda.mem_get_info(dev)[0]
        plan = stap.Plan([s.dims() for s in specs], device=dev, precision=prec,
                         max_workspace_bytes=max(0, free - (8 << 30)))
        t0 = time.perf_counter()
        plan.autotune(cubes, outs, reps=1)
        tune_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            plan.run_cpi(cubes, outs)
        torch.cuda.synchronize()
        times = time_steps(lambda: plan.run_cpi(cubes, outs), steps, flush, stream)
        code, failed = plan.status()
        if code != stap.STAP_OK:
            raise RuntimeError(f"batch {PREC_NAMES[prec]}: device status {code} ({failed} failed)")
        outs_pick[prec] = {i: outs[i][:, :, b * 64:(b + 1) * 64].cpu().numpy() for i, b in picks}
        ms = sum(times) / steps
        # the autotuner's schedule, and the other one timed beside it (2 steps)
        chosen = stap.stap_plan_get_batch_schedule(plan.handle)
        other = stap.STAP_BATCH_STREAMS if chosen == stap.STAP_BATCH_PERSISTENT else stap.STAP_BATCH_PERSISTENT
        sched_names = {stap.STAP_BATCH_PERSISTENT: "persistent", stap.STAP_BATCH_STREAMS: "streams"}
        schedules = {sched_names[chosen]: ms}
        try:
            plan.set_batch_schedule(other)
            plan.run_cpi(cubes, outs)
            torch.cuda.synchronize()
            t_other = time_steps(lambda: plan.run_cpi(cubes, outs), 2, flush, stream)
            schedules[sched_names[other]] = sum(t_other) / 2
            plan.set_batch_schedule(chosen)
        except Exception as exc:   # a side measurement must not lose the leg
            schedules[sched_names[other]] = f"{type(exc).__name__}: {exc}"[:200]
        log(f"batch {PREC_NAMES[prec]}: {ms:.1f} ms/step ({sched_names[chosen]}), schedules {schedules}")
        res["mixed" if prec else "fp32"] = {
            "precision": PREC_NAMES[prec], "arithmetic": PREC_TEXT[prec] + "; " + SOLVE_TEXT,
            "value": cells / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "autotune_s": tune_s,
            "schedule": sched_names[chosen], "ms_per_step_by_schedule": schedules,
            "gpu_launches_per_step": 4 * len(specs),
            "fp64_solve_frac_of_step": sum(solve_flops(s) for s in specs) / (ms * 1e-3) / 1e12 /
            peaks()["fp64_tflops"]}
        plan.close()
        del plan, outs
        torch.cuda.empty_cache()
    res["mixed_vs_fp32"] = res["mixed"]["value"] / res["fp32"]["value"]
    if not args.no_cpu_baseline:
        import oracle
        errs = {}
        for prec, got in outs_pick.items():
            num = den = worst = 0.0
            for i, b in picks:
                s = specs[i]
                key = (i, b)
                if key not in errs:
                    errs[key] = oracle.run(oracle.Dims(*s.dims()), cubes[i].cpu().numpy(), r0=b * 64,
                                           nr=64)["out"]
                ref = errs[key]
                num += float(np.sum((got[i].astype(np.float64) - ref) ** 2))
                den += float(np.sum(ref ** 2))
                worst = max(worst, power_errors(got[i], ref)["max_cell"])
            res.setdefault("errors_vs_oracle", {})[PREC_NAMES[prec]] = {
                "normwise": (num / den) ** 0.5, "max_cell": worst, "blocks": len(picks)}
    del cubes
    torch.cuda.empty_cache()
    return res


def run_batch(args):
    """The batch workload: 512 uneven CPIs through one stap_run_cpi call (a
    captured CUDA graph replayed each step).  Each rank processes its own
    batch (a different seed)."""
    import torch
    import torch.distributed as dist
    from paper_2203_06233_gb300 import stap, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = synth.batch_cpis(512, seed=4 + 1000 * rank)
    cubes = [synth.make_cube_torch(s, dev) for s in specs]
    outs = [torch.empty((s.n_steering, s.n_dop, s.n_range), dtype=torch.float32, device=dev)
            for s in specs]
    # workspace: as much of the all-concurrent size as free HBM allows (8 GiB spare)
    free = torch.cuda.mem_get_info(dev)[0]
    plan = stap.Plan([s.dims() for s in specs], device=dev, max_workspace_bytes=max(0, free - (8 << 30)))
    tuning = plan.autotune(cubes, outs)
    flushbuf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def flush():
        flushbuf.zero_()

    def step():
        plan.run_cpi(cubes, outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    code, failed = plan.status()
    if code != stap.STAP_OK:
        raise RuntimeError(f"device status {code} ({failed} failed systems) after warm-up")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = time_steps(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    cells = sum(s.cells for s in specs)
    total_ms, value = aggregate(sum(times), cells * args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    sf = sum(solve_flops(s, refine=1) for s in specs)
    pk = peaks()
    achieved = sf / (ms_per_step * 1e-3) / 1e12
    roofline = {"kernel": "all solve kernels of the batch (FP64)", "bound": "alu",
                "achieved": achieved, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                "frac": achieved / pk["fp64_tflops"], "traffic": None,
                "basis": "FP64 solve flops of all 512 CPIs / whole step time (a lower bound for "
                         "the solve kernels: the step also runs the other 1536 launches)",
                "peak_src": "FP64: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (unit count and max clock)"}

    # end to end: every cube from pinned host memory, every output back
    h2d = sum(c.numel() * 8 for c in cubes)
    d2h = sum(o.numel() * 4 for o in outs)
    e2e = None
    try:
        cubes_pin = [c.cpu().pin_memory() for c in cubes]
        outs_pin = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]

        def e2e_step():
            for c, cp in zip(cubes, cubes_pin):
                c.copy_(cp, non_blocking=True)
            plan.run_cpi(cubes, outs)
            for o, op in zip(outs, outs_pin):
                op.copy_(o, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e2e_ms = statistics.mean(time_steps(e2e_step, max(1, min(3, args.steps)), flush, stream))
        e2e = {"value": world * cells / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}
        del cubes_pin, outs_pin
    except RuntimeError as exc:   # pinned host memory exhausted
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "unavailable": f"pinned host buffers: {exc}"[:200]}
    shapes = {}
    for s in specs:
        key = f"C{s.n_chan} T{s.tdof} K{s.n_dop} S{s.n_steering}"
        shapes[key] = shapes.get(key, 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch of {len(specs)} uneven CPIs: C in {{4,8,16}}, T in {{2,3,4}}, "
                               f"P = K in {{64,128,256}}, R = 64 x U{{16..256}}, B 64, S in {{8,16}}",
                   "cells_per_step": cells, "n_cpi": len(specs), "distinct_shapes": len(shapes),
                   "workspace_gib": plan.workspace.numel() / 2 ** 30,
                   "batch_bytes_gib": plan.batch_bytes / 2 ** 30,
                   "precision": PREC_TEXT[0] + "; " + SOLVE_TEXT,
                   "l2": "inputs (47 GB of cubes) larger than L2; L2 also flushed between steps",
                   "tuned_shapes": len(tuning), "parallelism": "one batch per GPU per step"},
        "e2e": e2e,
        "gpu_launches": 4 * len(specs) * args.steps,
        "roofline": roofline,
        "clocks": clk.summary(),
    }
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_paper_cube(args):
    """The paper's cube shape (1000 channels, 100 pulses, 30000 samples, about
    24 GB) through the subarray front end (4 subarrays of 250 elements) and the
    chain (K128 T3 B100 S16).  value: element cube resident in HBM; e2e: every
    element cube streamed from pinned host memory (stap_run_stream), against
    the paper's real-time bar of 33.3 cubes/s."""
    import torch
    import torch.distributed as dist
    from paper_2203_06233_gb300 import stap, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    es = dataclasses.replace(synth.paper_cube_elements(), sub=rank)
    N, P, K, R, T, B, S = es.dims()
    C = synth.PAPER_CUBE_CHANNELS
    M = N // C
    W = (np.arange(N)[None, :] // M == np.arange(C)[:, None]).astype(np.complex128)
    plan = stap.Plan((C, P, K, R, T, B, S), device=dev, front_end=W)
    elem = synth.make_cube_torch(es, dev)                       # [N][P][R], 24 GB
    y = torch.empty((C, P, R), dtype=torch.complex64, device=dev)
    out = torch.empty((S, K, R), dtype=torch.float32, device=dev)
    tuning = plan.autotune(plan.reduce_channels(elem, y), out)
    nchunk = -(-N // max(1, plan_chunk(plan)))

    def step():
        plan.reduce_channels(elem, y)
        plan.run_cpi(y, out)

    def noflush():
        pass                                                     # inputs (24 GB) exceed L2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    code, failed = plan.status()
    if code != stap.STAP_OK:
        raise RuntimeError(f"paper cube: device status {code} ({failed} failed systems)")
    steps = max(3, min(args.steps, 200))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = time_steps(step, steps, noflush, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    cells = K * R
    total_ms, value = aggregate(sum(times), cells * steps, world, dev)
    ms_per_step = total_ms / steps
    red_ms = statistics.mean(time_steps(lambda: plan.reduce_channels(elem, y), max(3, steps // 4),
                                        noflush, stream))
    pk = peaks()
    red_bytes = 8.0 * N * P * R + 8.0 * C * P * R        # elements read once, reduced cube written once
    roofline = {"kernel": "reduce_channels_kernel (front end: 1000 elements -> 4 subarrays)",
                "bound": "hbm", "achieved": red_bytes / red_ms / 1e6, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": red_bytes / red_ms / 1e6 / pk["hbm_gbs"], "traffic": None,
                "peak_src": "MEASURED_PEAKS.json hbm_gbs (measured)"}

    # ---- end to end: element cubes streamed from pinned host memory ----
    e2e = None
    need = 2.5 * N * P * R * 8
    avail = host_mem_available()
    if avail is not None and avail >= need:
        host = torch.empty((N, P, R), dtype=torch.complex64, pin_memory=True)
        host.copy_(elem)
        del elem
        torch.cuda.empty_cache()
        host_outs = [torch.empty((S, K, R), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        plan.run_stream([host] * 2, host_outs)                   # warm-up, grows the workspace
        torch.cuda.synchronize()
        n_stream = max(4, min(args.steps, 20))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run_stream([host] * n_stream, [host_outs[i % 2] for i in range(n_stream)])
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms, _ = aggregate(e0.elapsed_time(e1), cells * n_stream, world, dev)
        e2e_ms /= n_stream
        e2e = {"value": world * cells / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": N * P * R * 8, "d2h_bytes_per_step": S * K * R * 4,
               "ms_per_step": e2e_ms, "cubes_per_s": world * 1e3 / e2e_ms,
               "api": f"stap_run_stream over {n_stream} element cubes from one pinned host cube: "
                      f"each copied in ({nchunk} chunks), reduced, run and its output copied out "
                      "inside the timed region"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"paper cube: N{N} elements P{P} R{R} (about {N * P * R * 8 / 1e9:.0f} GB), "
                               f"front end to C{C} subarrays of {M}, then K{K} T{T} B{B} S{S} (D={C*T}), "
                               "40 dB CNR per element, 8 targets",
                   "cells_per_step": cells, "l2": "not flushed: the 24 GB element cube exceeds L2",
                   "parallelism": "one cube per GPU per step", "tuning": tuning},
        "cubes_per_s": world * 1e3 / ms_per_step,
        "real_time_bar_cubes_per_s": 33.3,
        "e2e": e2e if e2e is not None else
        {"value": None, "unit": UNIT, "unavailable": f"host memory {avail} B below {need:.0f} B"},
        "gpu_launches": (1 + 4 * slab_count(tuning, R // B)) * steps,
        "roofline": roofline,
        "kernels_ms": {"front_end": red_ms, "chain": ms_per_step - red_ms},
        "clocks": clk.summary(),
    }
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def plan_chunk(plan):
    """Element rows per front-end chunk (the library's default: about 512 MB)."""
    P, R = plan.dims[0].n_pulses, plan.dims[0].n_range
    return max(1, min(plan.n_elem, (512 << 20) // (P * R * 8)))


def host_mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2203_06233_gb300", "csrc", "solve.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def run_reference(args):
    """The FP64 CPU oracle on the host cores, rank 0 only: each step one
    seeded range block of the workload (all eight steps on its window),
    cells/s over the steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2203_06233_gb300 import synth
    if NAME in ("batch", "paper_cube"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm covers the single-CPI "
                          f"workloads; {NAME} has none"}), flush=True)
        return
    spec = workload_spec(0, NAME)
    B, NB, K = spec.training_block, spec.NB, spec.n_dop
    cube = synth.make_cube(spec) if spec.cells <= (1 << 24) else None

    def window(b0, nb):   # large cubes: generate only the windows the steps read
        if cube is None:
            return synth.make_cube_window(spec, b0 * B, nb * B)
        return np.ascontiguousarray(cube[:, :, b0 * B:(b0 + nb) * B])

    # size each step (a range window of whole blocks) so the run ends in ~3 minutes
    w0 = window(0, 1)
    dw = oracle.Dims(spec.n_chan, spec.n_pulses, K, B, spec.tdof, B, spec.n_steering)
    oracle.run(dw, w0, r0=0, nr=B)          # first call: thread pool start-up
    t0 = time.perf_counter()
    oracle.run(dw, w0, r0=0, nr=B)
    per_block = time.perf_counter() - t0
    nblk = int(max(1, min(NB, 150.0 / max(1, args.steps + args.warmup) / max(per_block, 1e-6))))
    nr = nblk * B
    dn = oracle.Dims(spec.n_chan, spec.n_pulses, K, nr, spec.tdof, B, spec.n_steering)
    # the steps' input windows, generated before the timed region
    b0s = [min((i * nblk) % NB, NB - nblk) for i in range(args.warmup + args.steps)]
    wins = {b0: window(b0, nblk) for b0 in sorted(set(b0s))}

    def one(i):
        oracle.run(dn, wins[b0s[i]], r0=0, nr=nr)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(args.warmup + i)
    el = time.perf_counter() - t0
    value = args.steps * K * nr / el
    sample = (f"each step: a range window of {nblk} block(s) x {B} cells x {K} bins of the {NAME} "
              f"CPI, all eight oracle steps on the window (blocks are independent)")
    cfg = workload_config(spec)
    cfg["precision"] = "FP64 oracle (plain C, IEEE double), every step"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg, "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# configuration number -> workload: the standard CPI (D = 12), the D = 64 CPI,
# the 512-CPI batch and the large CPI (D = 128)
CONFIG_WORKLOADS = {2: "standard", 3: "mixed", 4: "batch", 5: "large"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-headline", action="store_true",
                    help="measure the headline workload only (no other workloads as keys)")
    ap.add_argument("--workload", choices=["large", "mixed", "mixed_small", "standard", "batch",
                                           "paper_cube"],
                    default="large",
                    help="large (the default) is the largest single-GPU CPI; batch: 512 uneven CPIs "
                         "per step in one graph replay; paper_cube: the paper's 1000-channel cube "
                         "through a subarray front end")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=None,
                    help="the workload by its configuration number: 2 standard, 3 mixed, 4 batch, "
                         "5 large (1, the small CPI, is a parity-test case in tests/, not a "
                         "benchmark workload)")
    args = ap.parse_args()
    if args.config is not None:
        if args.config not in CONFIG_WORKLOADS:
            ap.error("configuration 1 (the small CPI) is a parity-test case, not a benchmark workload")
        args.workload = CONFIG_WORKLOADS[args.config]
    global NAME
    NAME = args.workload
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != world:
        ap.error(f"--gpus {args.gpus} but {world} process(es): launch N > 1 GPUs with "
                 "torch.distributed.run (one process per GPU)")
    if args.impl == "reference":
        run_reference(args)
    elif NAME == "batch":
        run_batch(args)
    elif NAME == "paper_cube":
        run_paper_cube(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
