"""Batched stap_run_cpi: uneven CPIs packed into waves, forked streams,
captured in a CUDA graph and replayed."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import MIXED_NORM_BAR, MIXED_PRECISIONS, PLAIN_CELL_BAR, mixed_cell_bar, power_errors

pytestmark = pytest.mark.gpu


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


def _uneven(n=12, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        C = int(rng.choice([4, 8, 16]))
        T = int(rng.choice([2, 3, 4]))
        K = int(rng.choice([64, 128]))
        R = 64 * int(rng.integers(2, 17))
        S = int(rng.choice([8, 16]))
        out.append(synth.CPISpec(C, K, K, R, T, 64, S, cnr_db=float(rng.uniform(20, 40)),
                                 targets=synth.random_targets(seed, 2, R, K, S, sub=i + 1),
                                 seed=seed, sub=i + 1))
    return out


@pytest.mark.parametrize("schedule", [stap.STAP_BATCH_PERSISTENT, stap.STAP_BATCH_STREAMS],
                         ids=["persistent", "streams"])
def test_batch_equals_single_cpi_runs_across_waves_and_replays(schedule):
    """Both batch schedules -- persistent launches per phase over all the
    wave's CPIs, or each CPI's chain on a side stream -- give each CPI exactly
    the output of its own one-CPI run, in one wave and in one wave per CPI,
    on the captured launch and on graph replays."""
    specs = _uneven()
    cubes = [torch.from_numpy(synth.make_cube(s)).cuda() for s in specs]
    singles = []
    for s, c in zip(specs, cubes):
        p = stap.Plan(s.dims())
        singles.append(p.run_cpi(c).clone())
        p.close()
    full = stap.Plan([s.dims() for s in specs])                    # one wave
    tight = stap.Plan([s.dims() for s in specs], max_workspace_bytes=0)   # one CPI per wave
    for plan in (full, tight):
        plan.set_batch_schedule(schedule)
        outs = plan.run_cpi(cubes)                                 # capture + launch
        again = plan.run_cpi(cubes, outs)                          # graph replay
        torch.cuda.synchronize()
        for o, ref in zip(again, singles):
            assert torch.equal(o, ref)
        fresh = [torch.zeros_like(o) for o in outs]                # new buffers: recapture
        plan.run_cpi(cubes, fresh)
        torch.cuda.synchronize()
        for o, ref in zip(fresh, singles):
            assert torch.equal(o, ref)
        assert plan.status() == (stap.STAP_OK, 0)
    full.close()
    tight.close()


def test_full_batch_workload_on_sampled_cpis():
    """512 uneven CPIs (C in {4,8,16}, T in {2,3,4}, P = K in {64,128,256},
    R in 1024..16384, B 64, S in {8,16}) in one call, on the plain path and
    on every mixed-precision path; the oracle checks one seeded block of 8
    seeded CPIs, each block's oracle result serving every path."""
    specs = synth.batch_cpis(512)
    cubes = [synth.make_cube_torch(s, "cuda") for s in specs]
    rng = np.random.default_rng(4)
    picks = [(i, int(rng.integers(specs[i].NB)))
             for i in sorted(int(x) for x in rng.choice(len(specs), 8, replace=False))]
    refs = {}
    for i, b in picks:
        s = specs[i]
        B = s.training_block
        refs[i] = oracle.run(oracle.Dims(*s.dims()), cubes[i].cpu().numpy(), r0=b * B, nr=B)["out"]
    bad = []
    for pname, prec in [("plain", stap.STAP_PREC_FP32)] + MIXED_PRECISIONS:
        plan = stap.Plan([s.dims() for s in specs], precision=prec)
        outs = plan.run_cpi(cubes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.run_cpi(cubes, outs)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        cells = sum(s.cells for s in specs)
        print(f"{pname} batch of {len(specs)} CPIs: {el * 1e3:.1f} ms, {cells / el:.3e} cells/s, "
              f"workspace {plan.workspace.numel() / 2**30:.1f} GiB of {plan.batch_bytes / 2**30:.1f}")
        assert plan.status() == (stap.STAP_OK, 0)
        for i, b in picks:
            s = specs[i]
            B = s.training_block
            got = outs[i][:, :, b * B:(b + 1) * B].cpu().numpy()
            e_cell, e_norm = power_errors(got, refs[i])
            print(f"  {pname} cpi {i} {s.dims()} block {b}: max-cell/floor={e_cell:.3e} "
                  f"normwise={e_norm:.3e}")
            g = growth(s)
            if pname == "plain":
                ok = e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
            else:
                ok = e_norm <= MIXED_NORM_BAR and e_cell <= mixed_cell_bar(s)
            if not ok:
                bad.append((pname, i, e_cell, e_norm))
        plan.close()
        del outs
        torch.cuda.empty_cache()
    assert not bad, bad


def test_autotune_keeps_results_and_round_trips_through_the_cache(tmp_path):
    """Autotuning changes launch shapes only: the tuned plan reproduces the
    default plan's output bit for bit (up to the apply kernel's summation
    order, checked against the parity bar), and the JSON cache restores the
    same choices into a fresh plan."""
    specs = _uneven(6, seed=9) + [synth.standard_cpi()]
    cubes = [torch.from_numpy(synth.make_cube(s)).cuda() for s in specs]
    base = stap.Plan([s.dims() for s in specs])
    ref = [o.clone() for o in base.run_cpi(cubes)]
    cache = str(tmp_path / "tune.json")
    tuned = stap.Plan([s.dims() for s in specs])
    choices = tuned.autotune(cubes, cache_path=cache)
    assert len(choices) == len({tuned._tune_key(i) for i in range(len(specs))})
    outs = tuned.run_cpi(cubes)
    torch.cuda.synchronize()
    for s, o, r in zip(specs, outs, ref):
        e_cell, e_norm = power_errors(o.cpu().numpy(), r.cpu().numpy().astype(np.float64))
        assert e_norm <= 1e-5 and e_cell <= 1e-4, (s.dims(), e_cell, e_norm)
    again = stap.Plan([s.dims() for s in specs])
    again.autotune(cubes, cache_path=cache)             # from the cache, no timing
    for i in range(len(specs)):
        assert stap.stap_plan_get_tuning(again.handle, i) == stap.stap_plan_get_tuning(tuned.handle, i)
    assert tuned.status() == (stap.STAP_OK, 0)
    for p in (base, tuned, again):
        p.close()


@pytest.mark.parametrize("prec", [stap.STAP_PREC_FP32, stap.STAP_PREC_BF16X3], ids=["fp32", "bf16x3"])
def test_persistent_batch_with_options_equals_single_runs(prec):
    """Persistent batches with the launches that have no persistent form
    mixed in (tensor-core kernels, neighbour training, the mixed-precision
    refinement solve): still each CPI's own one-CPI output."""
    specs = _uneven(6, seed=11)
    cubes = [torch.from_numpy(synth.make_cube(s)).cuda() for s in specs]
    for kw in ({}, {"training": stap.STAP_TRAIN_NEIGHBOURS},
               {"solver": stap.STAP_SOLVE_MIXED_IR, "refine_steps": 2}):
        singles = []
        for s, c in zip(specs, cubes):
            p = stap.Plan(s.dims(), precision=prec, **kw)
            singles.append(p.run_cpi(c).clone())
            p.close()
        plan = stap.Plan([s.dims() for s in specs], precision=prec, **kw)
        plan.set_batch_schedule(stap.STAP_BATCH_PERSISTENT)
        outs = plan.run_cpi(cubes)
        again = plan.run_cpi(cubes, outs)
        torch.cuda.synchronize()
        for o, ref in zip(again, singles):
            assert torch.equal(o, ref), kw
        assert plan.status() == (stap.STAP_OK, 0)
        plan.close()
