"""Streamed runs (stap_run_stream): host cubes copied in, the chain, results
copied out, with the copies of neighbouring CPIs overlapping the chain.  Every
streamed result must equal stap_run_cpi on the same cube bit for bit."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2203_06233_gb300 import stap, synth

pytestmark = pytest.mark.gpu


def _cubes(spec, n):
    """n different cubes of one shape (the seed varies)."""
    return [torch.from_numpy(synth.make_cube(dataclasses.replace(spec, seed=spec.seed + 100 + i)))
            for i in range(n)]


def _reference(plan, cubes):
    return [plan.run_cpi(c.cuda()).cpu() for c in cubes]


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_streamed_results_equal_single_runs(pinned):
    spec = synth.small_cpi()
    cubes = _cubes(spec, 5)
    plan = stap.Plan(spec.dims())
    ref = _reference(plan, cubes)
    host = [c.pin_memory() if pinned else c.clone() for c in cubes]
    outs = None if pinned else [torch.empty(plan.shapes()["out"]) for _ in cubes]
    outs = plan.run_stream(host, outs)
    torch.cuda.current_stream().synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_streamed_standard_cpi_with_slabs_back_to_back_calls():
    spec = synth.standard_cpi()
    cubes = _cubes(spec, 4)
    plan = stap.Plan(spec.dims())
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[6] = 4                                   # four range slabs per chain
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    ref = _reference(plan, cubes)
    host = [c.pin_memory() for c in cubes]
    first = plan.run_stream(host[:3])
    second = plan.run_stream(host[1:])               # queued behind the first call
    torch.cuda.current_stream().synchronize()
    for o, r in zip(first, ref[:3]):
        assert torch.equal(o, r)
    for o, r in zip(second, ref[1:]):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_stream_of_zero_and_one_cpi():
    spec = synth.small_cpi()
    cubes = _cubes(spec, 1)
    plan = stap.Plan(spec.dims())
    ref = _reference(plan, cubes)
    assert plan.run_stream([]) == []
    out = plan.run_stream([cubes[0].pin_memory()])
    torch.cuda.current_stream().synchronize()
    assert torch.equal(out[0], ref[0])
    plan.close()


@pytest.mark.parametrize("opts", [dict(snapshots=stap.STAP_SNAP_PRI_STAGGERED),
                                  dict(training=stap.STAP_TRAIN_NEIGHBOURS),
                                  dict(solver=stap.STAP_SOLVE_MIXED_IR, refine_steps=2)],
                         ids=["staggered", "neighbours", "mixed_ir"])
def test_streamed_option_plans_equal_single_runs(opts):
    spec = synth.small_cpi()
    cubes = _cubes(spec, 3)
    plan = stap.Plan(spec.dims(), **opts)
    ref = _reference(plan, cubes)
    outs = plan.run_stream([c.pin_memory() for c in cubes])
    torch.cuda.current_stream().synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_stream_rejects_device_tensors_and_wrong_shapes():
    spec = synth.small_cpi()
    plan = stap.Plan(spec.dims())
    cube = torch.from_numpy(synth.make_cube(spec))
    with pytest.raises(TypeError):
        plan.run_stream([cube.cuda()])
    with pytest.raises(ValueError):
        plan.run_stream([cube[:, :, :128].contiguous()])
    plan.close()
