"""Run a few whole-CPI steps of one workload for a profiler.

    python -m paper_2203_06233_gb300.profile_step --workload standard --steps 5
    ncu --clock-control none --profile-from-start off -k regex:<kernel> -c 1 \
        python -m paper_2203_06233_gb300.profile_step ...

(--clock-control none leaves the GPU's clocks alone; capture one kernel and a
few launches at a time.)

Builds the plan, takes the launch choices from the autotune cache (timing them
on the device when the cache lacks the shape), warms up, and then runs
``--steps`` calls of ``stap_run_cpi`` between cudaProfilerStart and
cudaProfilerStop, so that a profiler started with profiling off sees exactly
the launches of those steps, and prints their mean time per step (CUDA
events on the current stream; no L2 flush between the steps).  The paper_cube workloads run the subarray front
end (1000 elements to 4 channels) before the chain in every step.  ``--slabs N`` overrides the tuned number of
range slabs (1 = the plain four-launch chain).  The input is the workload's
seeded synthetic cube, generated on the device.
"""
import argparse
import dataclasses

import numpy as np
import torch

from . import stap, synth

PRECISIONS = {"fp32": stap.STAP_PREC_FP32, "tf32x3": stap.STAP_PREC_TF32X3,
              "bf16x3": stap.STAP_PREC_BF16X3, "fp16s": stap.STAP_PREC_FP16_SCALED}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="standard",
                    choices=sorted(synth.WORKLOADS) + sorted(synth.ELEMENT_WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--slabs", type=int, default=0, help="override the tuned range slabs (0 = keep)")
    ap.add_argument("--solver", default="fp64", choices=["fp64", "mixed_ir"])
    ap.add_argument("--snapshots", default="adjacent", choices=["adjacent", "staggered"])
    ap.add_argument("--training", default="own", choices=["own", "neighbours"])
    ap.add_argument("--refine", type=int, default=None,
                    help="refinement steps (default: 1 for fp64, 2 for mixed_ir)")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    prec = PRECISIONS[a.precision]
    solver = stap.STAP_SOLVE_FP64 if a.solver == "fp64" else stap.STAP_SOLVE_MIXED_IR
    refine = a.refine if a.refine is not None else (1 if a.solver == "fp64" else 2)
    opts = dict(snapshots=stap.STAP_SNAP_PRI_STAGGERED if a.snapshots == "staggered"
                else stap.STAP_SNAP_ADJACENT_BINS,
                training=stap.STAP_TRAIN_NEIGHBOURS if a.training == "neighbours"
                else stap.STAP_TRAIN_OWN_BLOCK)
    elem = None
    if a.workload in synth.ELEMENT_WORKLOADS:
        # element cube through the subarray front end, then the chain
        es = synth.ELEMENT_WORKLOADS[a.workload]()
        N, P, K, R, T, B, S = es.dims()
        C = synth.PAPER_CUBE_CHANNELS
        W = (np.arange(N)[None, :] // (N // C) == np.arange(C)[:, None]).astype(np.complex128)
        spec = dataclasses.replace(es, n_chan=C)
        plan = stap.Plan(spec.dims(), device=dev, precision=prec, refine_steps=refine, solver=solver,
                         front_end=W, **opts)
        elem = synth.make_cube_torch(es, dev)
        cube = plan.reduce_channels(elem)
    else:
        spec = synth.WORKLOADS[a.workload]()
        if isinstance(spec, (list, tuple)):
            raise SystemExit("profile_step runs one-CPI workloads")
        cube = synth.make_cube_torch(spec, dev)
        plan = stap.Plan(spec.dims(), device=dev, precision=prec, refine_steps=refine, solver=solver,
                         **opts)
    out = torch.empty(plan.shapes(0)["out"], dtype=torch.float32, device=dev)
    tuning = plan.autotune(cube, out)
    if a.slabs > 0:
        choices = stap.stap_plan_get_tuning(plan.handle, 0)
        choices[6] = a.slabs
        stap.stap_plan_set_tuning(plan.handle, 0, choices)

    def step():
        if elem is not None:
            plan.reduce_channels(elem, cube)
        plan.run_cpi(cube, out)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    t0.record()
    for _ in range(a.steps):
        step()
    t1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = t0.elapsed_time(t1) / max(a.steps, 1)
    code, failed = plan.status()
    plan.close()
    print(f"{a.workload} {a.precision} {a.solver} refine {refine}: dims {spec.dims()}, tuning {tuning}, "
          f"slabs override {a.slabs}, {a.steps} steps, {ms:.3f} ms per step, status {code} ({failed} failed)")
    if code != stap.STAP_OK:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
