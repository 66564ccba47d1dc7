"""PRI-staggered snapshots (STAP_SNAP_PRI_STAGGERED): T sub-windows of
P - T + 1 pulses replace the T adjacent bins.  Parity of every step and of the
whole path with the oracle's oracle_doppler_staggered / oracle_run_staggered,
at the bars of the adjacent-bin path (tests/test_gpu_parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import (EPS32, MIXED_NORM_BAR, PLAIN_CELL_BAR, cell_bound, mixed_cell_bar, power_errors,
                     to_np)

pytestmark = pytest.mark.gpu

STAG = stap.STAP_SNAP_PRI_STAGGERED

SPECS = {
    "small": synth.small_cpi(),
    "standard": synth.standard_cpi(),
    "one_pulse_windows": synth.CPISpec(2, 4, 8, 64, 4, 16, 3, cnr_db=20.0, seed=41),      # T = P
    "even_T_ragged": synth.CPISpec(3, 20, 32, 96, 2, 32, 5, cnr_db=30.0, seed=42),        # D = 6
    "D64": synth.CPISpec(16, 32, 64, 256, 4, 64, 8, cnr_db=40.0, seed=43),               # per-CTA solve
}
IDS = list(SPECS)


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


def _dims(spec):
    return oracle.Dims(*spec.dims())


def _plan(spec, **kw):
    return stap.Plan(spec.dims(), snapshots=STAG, **kw)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dtype)


@pytest.mark.parametrize("name", IDS)
def test_staggered_doppler_matches_the_oracle(name):
    spec = SPECS[name]
    d = _dims(spec)
    cube = synth.make_cube(spec)
    ref = oracle.doppler_staggered(d, cube)
    plan = _plan(spec)
    dop = to_np(plan.doppler(_dev(cube, torch.complex64)))
    assert dop.shape == (spec.D, spec.n_dop, spec.n_range)
    tol = 2 * EPS32 * max(1, np.log2(spec.n_dop)) + 4 * EPS32
    for row in range(spec.D):
        err = np.linalg.norm(dop[row] - ref[row]) / np.linalg.norm(ref[row])
        assert err <= tol, (row, err, tol)
    plan.close()


@pytest.mark.parametrize("name", IDS)
def test_staggered_covariance_matches_the_oracle(name):
    spec = SPECS[name]
    d = _dims(spec)
    e = oracle.staggered_dims(d)
    dop64 = oracle.doppler_staggered(d, synth.make_cube(spec)).astype(np.complex64)
    ref = oracle.covariance(e, dop64)
    plan = _plan(spec)
    cov = to_np(plan.covariance(_dev(dop64, torch.complex64)))
    np.testing.assert_array_equal(cov, np.conj(np.swapaxes(cov, -1, -2)))
    num = np.linalg.norm((cov - ref).reshape(spec.n_dop, spec.NB, -1), axis=-1)
    den = np.linalg.norm(ref.reshape(spec.n_dop, spec.NB, -1), axis=-1)
    assert np.max(num / den) <= 1e-10, np.max(num / den)
    plan.close()


@pytest.mark.parametrize("name", IDS)
def test_staggered_weights_use_the_staggered_steering(name):
    spec = SPECS[name]
    d = _dims(spec)
    e = oracle.staggered_dims(d)
    cov = oracle.covariance(e, oracle.doppler_staggered(d, synth.make_cube(spec)))
    ref, _, nf = oracle.weights(e, cov, oracle.default_steering_staggered(d))
    assert nf == 0
    plan = _plan(spec)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    assert plan.status() == (stap.STAP_OK, 0)
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2), np.max(err)
    plan.close()


@pytest.mark.parametrize("name", IDS)
def test_staggered_apply_matches_the_oracle(name):
    spec = SPECS[name]
    d = _dims(spec)
    e = oracle.staggered_dims(d)
    dop = oracle.doppler_staggered(d, synth.make_cube(spec))
    w, _, _ = oracle.weights(e, oracle.covariance(e, dop), oracle.default_steering_staggered(d))
    dop64, w64 = dop.astype(np.complex64), w.astype(np.complex64)
    ref = oracle.apply(e, dop64, w64)
    plan = _plan(spec)
    out = to_np(plan.apply(_dev(dop64, torch.complex64), _dev(w64, torch.complex64)))
    bound = cell_bound(dop64, w64, 1, spec.training_block)     # one bin per snapshot
    viol = np.abs(out - ref) > bound
    assert not viol.any(), (int(viol.sum()), float(np.max(np.abs(out - ref) - bound)))
    plan.close()


@pytest.mark.parametrize("solver", [stap.STAP_SOLVE_FP64, stap.STAP_SOLVE_MIXED_IR],
                         ids=["fp64", "mixed_ir"])
@pytest.mark.parametrize("name", IDS)
def test_staggered_run_cpi_end_to_end(name, solver):
    spec = SPECS[name]
    d = _dims(spec)
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube, staggered=True)["out"]
    plan = _plan(spec, solver=solver, refine_steps=2 if solver == stap.STAP_SOLVE_MIXED_IR else 1)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    g = growth(spec)
    print(f"{name}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e} (x{g:.2f})")
    assert e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
    plan.close()


@pytest.mark.parametrize("name", ["standard", "D64"])
def test_staggered_mixed_precision_end_to_end(name):
    """3xTF32 tensor-core covariance and apply with staggered snapshots: the
    mixed bar, normwise <= 1e-3 (grown as for the plain path)."""
    spec = SPECS[name]
    d = _dims(spec)
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube, staggered=True)["out"]
    plan = _plan(spec, precision=stap.STAP_PREC_TF32X3)
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[5], choices[8] = 3, 2                   # tensor-core apply and covariance
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    print(f"{name} mixed: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= MIXED_NORM_BAR and e_cell <= mixed_cell_bar(spec), (e_cell, e_norm)
    plan.close()


def test_staggered_steps_compose_slabs_agree_and_runs_are_deterministic():
    spec = SPECS["standard"]
    cube = _dev(synth.make_cube(spec), torch.complex64)
    plan = _plan(spec)
    run = plan.run_cpi(cube).clone()
    dop = plan.doppler(cube)
    steps = plan.apply(dop, plan.solve_weights(plan.covariance(dop)))
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[6] = 4                                  # four range slabs on their own streams
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    slabbed = plan.run_cpi(cube).clone()
    again = plan.run_cpi(cube)
    torch.cuda.synchronize()
    assert torch.equal(run, steps) and torch.equal(run, slabbed) and torch.equal(run, again)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_staggered_batch_equals_single_runs():
    specs = [SPECS["small"], SPECS["one_pulse_windows"], SPECS["even_T_ragged"], SPECS["small"]]
    cubes = [_dev(synth.make_cube(s), torch.complex64) for s in specs]
    singles = []
    for s, c in zip(specs, cubes):
        p = _plan(s)
        singles.append(p.run_cpi(c).clone())
        p.close()
    plan = stap.Plan([s.dims() for s in specs], snapshots=STAG)
    outs = plan.run_cpi(cubes)
    again = plan.run_cpi(cubes, outs)               # graph replay
    torch.cuda.synchronize()
    for o, r in zip(again, singles):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_staggered_with_neighbour_training_matches_the_oracle():
    spec = SPECS["small"]
    d = _dims(spec)
    e = oracle.staggered_dims(d)
    cube = synth.make_cube(spec)
    dop = oracle.doppler_staggered(d, cube)
    trn = oracle.train_neighbours(e, oracle.covariance(e, dop))
    w, _, nf = oracle.weights(e, trn, oracle.default_steering_staggered(d))
    assert nf == 0
    ref = oracle.apply(e, dop, w)
    plan = _plan(spec, training=stap.STAP_TRAIN_NEIGHBOURS)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    assert e_norm <= 1e-5 and e_cell <= PLAIN_CELL_BAR
    plan.close()


def test_staggered_with_one_dof_is_the_adjacent_bin_path_on_the_gpu():
    spec = synth.CPISpec(4, 16, 16, 64, 1, 16, 4, cnr_db=25.0, seed=44)   # T = 1
    cube = _dev(synth.make_cube(spec), torch.complex64)
    a = stap.Plan(spec.dims())
    s = _plan(spec)
    assert torch.equal(a.doppler(cube), s.doppler(cube))
    assert torch.equal(a.run_cpi(cube), s.run_cpi(cube))
    a.close()
    s.close()


def test_staggered_target_recovered_on_gpu():
    spec = SPECS["small"]
    out = to_np(_plan(spec).run_cpi(_dev(synth.make_cube(spec), torch.complex64)))
    assert int(np.argmax(out[2, 24])) == 128
    assert 10 * np.log10(out[2, 24, 128] / np.median(out)) > 10.0
