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

from _parity import PLAIN_CELL_BAR, power_errors


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


def _cases():
    """(spec, options, option kwargs of the workspace plan, oracle kwargs):
    the default path on two different CPIs, the tensor-core (3xTF32) path on
    a D = 64 CPI and PRI-staggered snapshots, each within the scratch limit
    and each with its own table and intermediate layout."""
    small, other = _noalloc_dims()
    d64 = synth.CPISpec(16, 32, 64, 256, 4, 128, 8, cnr_db=40.0, seed=14)
    o_tc = stap.stap_options_default()
    o_tc.precision = stap.STAP_PREC_TF32X3
    o_st = stap.stap_options_default()
    o_st.snapshots = stap.STAP_SNAP_PRI_STAGGERED
    return [(small, None, {}, {}), (other, None, {}, {}),
            (d64, o_tc, {"precision": stap.STAP_PREC_TF32X3}, None),
            (small, o_st, {"snapshots": stap.STAP_SNAP_PRI_STAGGERED}, {"staggered": True})]


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    """Each case through stap_run_cpi_noalloc, twice in a row and after the
    other cases (so every call meets scratch that an earlier, differently laid
    out call left behind), equals stap_run_cpi with a caller workspace bit for
    bit: both run the same kernels with the same default launch choices.  The
    small CPI is also checked against the oracle, and device memory stays
    unchanged across the no-allocation calls."""
    import torch
    import oracle
    cases = _cases()
    for s, _, _, _ in cases:
        h, run_bytes = stap.stap_plan_create([s.dims()])
        stap.stap_plan_destroy(h)
        assert run_bytes <= stap.STAP_NOALLOC_SCRATCH_BYTES
    cubes = [torch.from_numpy(synth.make_cube(s)).to("cuda") for s, _, _, _ in cases]
    refs = []
    for (s, _, kw, _), c in zip(cases, cubes):
        plan = stap.Plan(s.dims(), device="cuda", **kw)
        refs.append(plan.run_cpi(c).clone())
        plan.close()
    outs = [torch.full((s.n_steering, s.n_dop, s.n_range), float("nan"), dtype=torch.float32,
                       device="cuda") for s, _, _, _ in cases]

    def call(i):
        s, opts, _, _ = cases[i]
        outs[i].fill_(float("nan"))
        failed = stap.stap_run_cpi_noalloc(s.dims(), cubes[i], outs[i], opts=opts, want_status=True)
        torch.cuda.synchronize()
        assert failed == 0
        assert torch.equal(outs[i], refs[i]), i

    for i in range(len(cases)):          # first call on every path (lazy module loading)
        call(i)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for i in (0, 0, 1, 1, 2, 2, 3, 3, 0, 2):
        call(i)
    assert torch.cuda.mem_get_info()[0] == free_before
    for i in (0, 3):                     # against the oracle as well
        s, _, _, okw = cases[i]
        ref = oracle.run(oracle.Dims(*s.dims()), synth.make_cube(s), **okw)["out"]
        e_cell, e_norm = power_errors(outs[i].cpu().numpy(), ref)
        assert e_norm <= 1e-5 and e_cell <= PLAIN_CELL_BAR, (i, e_cell, e_norm)
