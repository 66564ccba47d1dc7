"""Training with guard cells.  STAP_TRAIN_NEIGHBOURS: block b's weights from
the mean of the covariances of blocks b-1 and b+1.  STAP_TRAIN_WINDOW: group
j's weights (B cells per group; B = 1 is a window per cell) from the groups
j-g-h .. j-g-1 and j+g+1 .. j+g+h beyond a guard band of g groups.  Parity
with the oracle's oracle_train_neighbours / oracle_run_neighbours and
oracle_train_window / oracle_run_window."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import PLAIN_CELL_BAR, power_errors, to_np

pytestmark = pytest.mark.gpu

NBR = stap.STAP_TRAIN_NEIGHBOURS


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


SPECS = {
    "small": synth.small_cpi(),
    "standard": synth.standard_cpi(),
    "two_blocks": synth.CPISpec(3, 20, 32, 64, 2, 32, 5, cnr_db=30.0, seed=31),        # NB = 2
    "D64": synth.CPISpec(16, 32, 64, 256, 4, 64, 8, cnr_db=40.0, seed=32),            # NB = 4
}


@pytest.mark.parametrize("name", list(SPECS))
def test_training_matrices_equal_the_oracle_bit_for_bit(name):
    spec = SPECS[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, synth.make_cube(spec)))
    ref = oracle.train_neighbours(d, cov)
    plan = stap.Plan(spec.dims(), training=NBR)
    got = plan.train_neighbours(torch.from_numpy(cov).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    plan.close()


@pytest.mark.parametrize("solver", [stap.STAP_SOLVE_FP64, stap.STAP_SOLVE_MIXED_IR],
                         ids=["fp64", "mixed_ir"])
@pytest.mark.parametrize("name", list(SPECS))
def test_run_cpi_with_neighbour_training_matches_the_oracle(name, solver):
    spec = SPECS[name]
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube, training=1)["out"]
    plan = stap.Plan(spec.dims(), training=NBR, solver=solver,
                     refine_steps=2 if solver == stap.STAP_SOLVE_MIXED_IR else 1)
    out = to_np(plan.run_cpi(torch.from_numpy(cube).cuda()))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    print(f"{name}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    g = growth(spec)
    assert e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
    plan.close()


def test_steps_compose_to_the_run_and_tuning_keeps_one_slab():
    spec = SPECS["standard"]
    cube = torch.from_numpy(synth.make_cube(spec)).cuda()
    plan = stap.Plan(spec.dims(), training=NBR)
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[6] = 4                                   # slabs: ignored with neighbour training
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    run = plan.run_cpi(cube).clone()
    dop = plan.doppler(cube)
    wts = plan.solve_weights(plan.train_neighbours(plan.covariance(dop)))
    steps = plan.apply(dop, wts)
    torch.cuda.synchronize()
    assert torch.equal(run, steps)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_batch_with_neighbour_training_equals_single_runs():
    specs = [SPECS["small"], SPECS["two_blocks"], SPECS["D64"], SPECS["small"]]
    cubes = [torch.from_numpy(synth.make_cube(s)).cuda() for s in specs]
    singles = []
    for s, c in zip(specs, cubes):
        p = stap.Plan(s.dims(), training=NBR)
        singles.append(p.run_cpi(c).clone())
        p.close()
    plan = stap.Plan([s.dims() for s in specs], training=NBR)
    outs = plan.run_cpi(cubes)
    again = plan.run_cpi(cubes, outs)                # graph replay
    torch.cuda.synchronize()
    for o, r in zip(again, singles):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_target_leaves_its_own_training_on_the_gpu():
    """As in the oracle pin: the small workload's target, trained on the
    neighbouring blocks, stands over four times higher above the median."""
    spec = SPECS["small"]
    cube = torch.from_numpy(synth.make_cube(spec)).cuda()
    own = to_np(stap.Plan(spec.dims()).run_cpi(cube))
    nbr = to_np(stap.Plan(spec.dims(), training=NBR).run_cpi(cube))
    assert int(np.argmax(nbr[2, 24])) == 128
    assert nbr[2, 24, 128] / np.median(nbr) > 4 * own[2, 24, 128] / np.median(own)


WIN = stap.STAP_TRAIN_WINDOW

# (spec, guard groups, training groups per side)
WINDOW_CASES = {
    "small_per_cell": (synth.CPISpec(4, 32, 32, 256, 3, 1, 4, cnr_db=30.0,
                                     targets=(synth.Target(128, 24, 2, 10.0, 0.0),), seed=1), 2, 16),
    "groups_of_4": (synth.CPISpec(3, 20, 32, 96, 2, 4, 5, cnr_db=30.0, seed=33), 1, 3),
    "neighbour_form": (synth.CPISpec(3, 20, 32, 64, 2, 16, 5, cnr_db=30.0, seed=34), 0, 1),
    "D64_per_8": (synth.CPISpec(16, 32, 64, 256, 4, 8, 8, cnr_db=40.0, seed=32), 1, 8),
}


@pytest.mark.parametrize("name", list(WINDOW_CASES))
def test_window_training_matrices_equal_the_oracle_bit_for_bit(name):
    spec, guard, half = WINDOW_CASES[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, synth.make_cube(spec)))
    ref = oracle.train_window(d, cov, guard, half)
    plan = stap.Plan(spec.dims(), training=WIN, train_guard=guard, train_half=half)
    got = plan.train_window(torch.from_numpy(cov).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    plan.close()


@pytest.mark.parametrize("name", list(WINDOW_CASES))
def test_run_cpi_with_window_training_matches_the_oracle(name):
    spec, guard, half = WINDOW_CASES[name]
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube, training=2, guard=guard, half=half)["out"]
    plan = stap.Plan(spec.dims(), training=WIN, train_guard=guard, train_half=half)
    out = to_np(plan.run_cpi(torch.from_numpy(cube).cuda()))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    print(f"{name} window: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    g = growth(spec)
    assert e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
    plan.close()


def test_per_cell_window_keeps_the_small_workload_target_unnulled():
    """The per-cell window (B = 1, 2 guard cells and 16 training cells on each
    side) on the small workload: the target is its row's maximum and stands
    far higher above the median than with the paper's own-block training."""
    spec, guard, half = WINDOW_CASES["small_per_cell"]
    cube = torch.from_numpy(synth.make_cube(spec)).cuda()
    win = stap.Plan(spec.dims(), training=WIN, train_guard=guard, train_half=half)
    own = stap.Plan(synth.small_cpi().dims())
    P_win = to_np(win.run_cpi(cube))
    P_own = to_np(own.run_cpi(cube))
    r_win = P_win[2, 24, 128] / np.median(P_win)
    r_own = P_own[2, 24, 128] / np.median(P_own)
    print(f"target over median: own block {r_own:.1f}, per-cell window {r_win:.1f}")
    assert int(np.argmax(P_win[2, 24])) == 128
    assert r_win > 4 * r_own
