"""The no-allocation entry point, stap_run_cpi_noalloc.

It serves callers that must not allocate device memory (a real-time loop that
forbids cudaMalloc after start-up, or an application whose own pool owns all
device memory): instead of a caller workspace it uses a fixed 16 MiB scratch
array inside the library.  These tests call it through the C ABI and check it
against the workspace entry point, stap_run_cpi, on consecutive calls that
share that array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_06233_gb300 import stap, synth

from _parity import power_errors


def _noalloc_dims():
    # two different CPIs, both within the scratch limit
    return [synth.small_cpi(),
            synth.CPISpec(3, 20, 32, 96, 2, 32, 5, cnr_db=30.0,
                          targets=(synth.Target(50, 3, 1, 12.0),), seed=11)]


def test_noalloc_rejects_cpi_larger_than_its_scratch_without_touching_cuda():
    L = stap.lib()
    big = stap.stap_dims(*synth.standard_cpi().dims())        # needs ~84 MB of scratch
    fake = ctypes.c_void_p(0x10000)                           # never dereferenced
    code = L.stap_run_cpi_noalloc(ctypes.byref(big), None, None, fake, fake, None)
    assert code == stap.STAP_ERR_NO_WORKSPACE
    h, run_bytes = stap.stap_plan_create([big])
    stap.stap_plan_destroy(h)
    assert run_bytes > stap.STAP_NOALLOC_SCRATCH_BYTES
    for spec in _noalloc_dims():
        h, run_bytes = stap.stap_plan_create([spec.dims()])
        stap.stap_plan_destroy(h)
        assert run_bytes <= stap.STAP_NOALLOC_SCRATCH_BYTES
    assert L.stap_run_cpi_noalloc(None, None, None, fake, fake, None) == stap.STAP_ERR_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    import torch
    specs = _noalloc_dims()
    cubes = [torch.from_numpy(synth.make_cube(s)).to("cuda") for s in specs]
    # the workspace entry point, as the reference for each CPI
    refs = []
    for s, c in zip(specs, cubes):
        plan = stap.Plan(s.dims(), device="cuda")
        refs.append(plan.run_cpi(c).cpu().numpy())
        plan.close()
    # two calls in a row on different CPIs (the second reuses the scratch the
    # first left behind), then the first CPI again
    for i in (0, 1, 0):
        s, c = specs[i], cubes[i]
        out = torch.full(tuple((s.n_steering, s.n_dop, s.n_range)), float("nan"),
                         dtype=torch.float32, device="cuda")
        failed = stap.stap_run_cpi_noalloc(s.dims(), c, out, want_status=True)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert failed == 0
        e_cell, e_norm = power_errors(got, refs[i].astype(np.float64))
        assert e_norm <= 1e-5 and e_cell <= 1e-3, (i, e_cell, e_norm)
