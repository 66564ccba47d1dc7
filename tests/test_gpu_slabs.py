"""One-CPI stap_run_cpi pipelined over range slabs: each slab's chain runs on
its own prioritised stream with its own covariance and weight region.  Every
per-cell result is computed exactly as in the unslabbed run, so the outputs
must agree bit for bit; the oracle check ties the slabbed run to Eq. 1-4."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import PLAIN_CELL_BAR, power_errors

pytestmark = pytest.mark.gpu


def _ragged():
    # NB = 13 blocks: no slab count above 1 divides it
    return synth.CPISpec(8, 64, 64, 13 * 64, 3, 64, 8, cnr_db=30.0,
                         targets=synth.random_targets(5, 2, 13 * 64, 64, 8, sub=3), seed=5, sub=3)


def _wide():
    return synth.CPISpec(32, 64, 64, 6 * 64, 4, 64, 4, cnr_db=30.0,      # D = 128, NB = 6
                         targets=synth.random_targets(6, 1, 6 * 64, 64, 4, sub=4), seed=6, sub=4)


SPECS = {"small": synth.small_cpi(), "standard": synth.standard_cpi(), "ragged": _ragged(),
         "wide": _wide()}


def _run(spec, cube, slabs, precision):
    plan = stap.Plan(spec.dims(), precision=precision)
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[6] = slabs
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    out = plan.run_cpi(cube).clone()
    again = plan.run_cpi(cube).clone()          # the slab streams are reused
    torch.cuda.synchronize()
    status = plan.status()
    plan.close()
    return out, again, status


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("precision", [stap.STAP_PREC_FP32, stap.STAP_PREC_TF32X3])
def test_slabbed_run_equals_unslabbed(name, precision):
    spec = SPECS[name]
    cube = torch.from_numpy(synth.make_cube(spec)).cuda()
    ref, _, st = _run(spec, cube, 1, precision)
    assert st == (stap.STAP_OK, 0)
    for slabs in (2, 3, 8, 64):                 # 64: clamped to min(8, NB)
        out, again, st = _run(spec, cube, slabs, precision)
        assert st == (stap.STAP_OK, 0), slabs
        assert torch.equal(out, ref), (name, slabs)
        assert torch.equal(again, ref), (name, slabs)


def test_slabbed_run_matches_oracle():
    spec = SPECS["ragged"]
    cube_np = synth.make_cube(spec)
    out, _, st = _run(spec, torch.from_numpy(cube_np).cuda(), 3, stap.STAP_PREC_FP32)
    assert st == (stap.STAP_OK, 0)
    d = oracle.Dims(*spec.dims())
    ref = oracle.run(d, cube_np)["out"]
    e_cell, e_norm = power_errors(out.cpu().numpy(), ref)
    print(f"slabs: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= 1e-5 and e_cell <= PLAIN_CELL_BAR, (e_cell, e_norm)


def test_one_cpi_autotune_picks_a_slab_count(tmp_path):
    spec = synth.standard_cpi()
    cube = torch.from_numpy(synth.make_cube(spec)).cuda()
    base = stap.Plan(spec.dims())
    ref = base.run_cpi(cube).clone()
    cache = str(tmp_path / "tune.json")
    plan = stap.Plan(spec.dims())
    choices = plan.autotune(cube, cache_path=cache)
    (key, tuning), = choices.items()
    assert key.endswith(" R%d" % spec.n_range)
    assert len(tuning) == stap.STAP_TUNING_LEN and tuning[6] in (1, 2, 4, 8)
    out = plan.run_cpi(cube)
    torch.cuda.synchronize()
    e_cell, e_norm = power_errors(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64))
    assert e_norm <= 1e-5 and e_cell <= 1e-4, (e_cell, e_norm)
    assert plan.status() == (stap.STAP_OK, 0)
    base.close()
    plan.close()
