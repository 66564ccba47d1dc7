"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every comparison uses the same seeded complex64 input on both sides; the
oracle never sees a value produced by the CUDA path.  Tolerances:

* Doppler (FP32 FFT): normwise relative error per channel <= 2 u log2(K) + 4u
  (FFT error bound with correctly rounded twiddles, u = 2^-24).
* Covariance (error-free FP32-pair accumulation, FP64 result): relative
  Frobenius error per system <= 1e-10 (Dot2 bound (2Bu)^2 plus FP64 rounding),
  Hermitian bit-exact.
* Weights (FP64 solve, complex64 result): relative 2-norm per vector <= 2u.
* Apply (FP32): every cell within the forward-error bound of the FP32 dot
  product (tests/_parity.cell_bound).
* Whole path, plain FP32: ||P - P_ref||_2 / ||P_ref||_2 <= 1e-5, and every
  cell within 1e-3 of max(P_ref, median P_ref), for D <= 12 (the plain
  workloads); for larger D both bars grow with the FP32 dot-product error
  of the apply, by (D + 2) / 14.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import EDGE_SPECS, EPS32, PLAIN_CELL_BAR, cell_bound, power_errors, to_np

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _cube(spec):
    return synth.make_cube(spec)


def _plan(spec, **kw):
    return stap.Plan(spec.dims(), device=DEV, **kw)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


SPECS = [synth.small_cpi(), synth.standard_cpi()] + EDGE_SPECS


def growth(spec):
    """End-to-end bars scale with the FP32 dot-product error of the apply,
    gamma_D ~ (D + 2) u, relative to the D = 12 of the plain workloads:
    1e-5 / 1e-3 hold as stated for D <= 12."""
    return max(1.0, (spec.D + 2) / 14.0)
IDS = ["small", "standard"] + [f"edge{i}" for i in range(len(EDGE_SPECS))]


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_doppler_parity(spec):
    d = oracle.Dims(*spec.dims())
    cube = _cube(spec)
    ref = oracle.doppler(d, cube)
    plan = _plan(spec)
    dop = to_np(plan.doppler(_dev(cube, torch.complex64)))
    K = spec.n_dop
    tol = 2 * EPS32 * max(1, np.log2(K)) + 4 * EPS32
    for c in range(spec.n_chan):
        err = np.linalg.norm(dop[c] - ref[c]) / np.linalg.norm(ref[c])
        assert err <= tol, (c, err, tol)


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_covariance_parity(spec):
    d = oracle.Dims(*spec.dims())
    dop64 = oracle.doppler(d, _cube(spec)).astype(np.complex64)     # same c64 input both sides
    ref = oracle.covariance(d, dop64)
    plan = _plan(spec)
    cov = to_np(plan.covariance(_dev(dop64, torch.complex64)))
    np.testing.assert_array_equal(cov, np.conj(np.swapaxes(cov, -1, -2)))
    num = np.linalg.norm((cov - ref).reshape(spec.n_dop, spec.NB, -1), axis=-1)
    den = np.linalg.norm(ref.reshape(spec.n_dop, spec.NB, -1), axis=-1)
    assert np.max(num / den) <= 1e-10, np.max(num / den)


def test_covariance_parity_with_subnormal_error_terms():
    """A Doppler cube scaled by 1e-16: the products are near 1e-32, so the
    error terms of the float pairs fall into FP32's subnormal range while
    their high parts stay normal; both convert exactly to FP64."""
    spec = synth.small_cpi()
    d = oracle.Dims(*spec.dims())
    dop64 = (oracle.doppler(d, _cube(spec)) * 1e-16).astype(np.complex64)
    ref = oracle.covariance(d, dop64)
    cov = to_np(_plan(spec).covariance(_dev(dop64, torch.complex64)))
    num = np.linalg.norm((cov - ref).reshape(spec.n_dop, spec.NB, -1), axis=-1)
    den = np.linalg.norm(ref.reshape(spec.n_dop, spec.NB, -1), axis=-1)
    assert np.max(num / den) <= 1e-10, np.max(num / den)


def test_covariance_of_an_infinite_sample_is_not_finite_where_the_oracle_is_not():
    spec = synth.small_cpi()
    d = oracle.Dims(*spec.dims())
    dop64 = oracle.doppler(d, _cube(spec)).astype(np.complex64)
    dop64[1, 7, 40] = np.inf
    with np.errstate(invalid="ignore", over="ignore"):
        ref = oracle.covariance(d, dop64)
    cov = to_np(_plan(spec).covariance(_dev(dop64, torch.complex64)))
    bad_ref = ~np.isfinite(ref.real) | ~np.isfinite(ref.imag)
    bad = ~np.isfinite(cov.real) | ~np.isfinite(cov.imag)
    # entries of the systems that never saw the sample stay finite and exact to 1e-10
    hit = bad_ref.reshape(spec.n_dop, spec.NB, -1).any(axis=-1)
    assert hit.any() and not hit.all()
    assert np.array_equal(bad.reshape(spec.n_dop, spec.NB, -1).any(axis=-1), hit)
    ok = ~hit
    num = np.linalg.norm((cov - ref).reshape(spec.n_dop, spec.NB, -1)[ok], axis=-1)
    den = np.linalg.norm(ref.reshape(spec.n_dop, spec.NB, -1)[ok], axis=-1)
    assert np.max(num / den) <= 1e-10


@pytest.mark.parametrize("refine", [0, 1, 2])
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_solve_weights_parity(spec, refine):
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))     # FP64 input both sides
    ref, status, nf = oracle.weights(d, cov)
    assert nf == 0
    plan = _plan(spec, refine_steps=refine)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2), np.max(err)
    assert plan.status() == (stap.STAP_OK, 0)


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_apply_parity(spec):
    d = oracle.Dims(*spec.dims())
    dop = oracle.doppler(d, _cube(spec))
    w, _, _ = oracle.weights(d, oracle.covariance(d, dop))
    dop64, w64 = dop.astype(np.complex64), w.astype(np.complex64)   # same c64 inputs both sides
    ref = oracle.apply(d, dop64, w64)
    plan = _plan(spec)
    out = to_np(plan.apply(_dev(dop64, torch.complex64), _dev(w64, torch.complex64)))
    bound = cell_bound(dop64, w64, spec.tdof, spec.training_block)
    viol = np.abs(out - ref) > bound
    assert not viol.any(), (int(viol.sum()), float(np.max(np.abs(out - ref) - bound)))


@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_run_cpi_end_to_end(spec):
    d = oracle.Dims(*spec.dims())
    cube = _cube(spec)
    ref = oracle.run(d, cube)["out"]
    plan = _plan(spec)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    e_cell, e_norm = power_errors(out, ref)
    g = growth(spec)
    print(f"dims={spec.dims()} max-cell/floor={e_cell:.3e} normwise={e_norm:.3e} (x{g:.2f})")
    assert e_norm <= 1e-5 * g, e_norm
    assert e_cell <= PLAIN_CELL_BAR * g, e_cell
    assert plan.status() == (stap.STAP_OK, 0)


def test_run_cpi_equals_step_by_step_and_is_deterministic():
    spec = synth.standard_cpi()
    cube = _dev(_cube(spec), torch.complex64)
    plan = _plan(spec)
    a = plan.run_cpi(cube)
    b = plan.run_cpi(cube)
    dop = plan.doppler(cube)
    steps = plan.apply(dop, plan.solve_weights(plan.covariance(dop)))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a, steps)


def test_small_workload_target_recovered_on_gpu():
    spec = synth.small_cpi()
    out = to_np(_plan(spec).run_cpi(_dev(_cube(spec), torch.complex64)))
    assert int(np.argmax(out[2, 24])) == 128
    assert 10 * np.log10(out[2, 24, 128] / np.median(out)) > 10.0


def test_user_steering_override():
    spec = synth.CPISpec(3, 16, 32, 128, 2, 32, 6, cnr_db=30.0, seed=31)
    d = oracle.Dims(*spec.dims())
    rng = np.random.default_rng(3)
    steer = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    cube = _cube(spec)
    ref = oracle.run(d, cube, steer=steer)["out"]
    plan = _plan(spec)
    plan.set_steering(steer)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    e_cell, e_norm = power_errors(out, ref)
    print(f"steering override: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= 1e-5 and e_cell <= 1e-3, (e_cell, e_norm)


@pytest.mark.parametrize("lf", [0.0, 1e-2, 0.3])
def test_load_factor_parity(lf):
    spec = synth.CPISpec(4, 32, 32, 256, 3, 64, 4, cnr_db=20.0, seed=41)
    d = oracle.Dims(*spec.dims())
    cube = _cube(spec)
    ref = oracle.run(d, cube, load_factor=lf)["out"]
    out = to_np(_plan(spec, load_factor=lf).run_cpi(_dev(cube, torch.complex64)))
    e_cell, e_norm = power_errors(out, ref)
    print(f"load factor {lf}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= 1e-5 and e_cell <= 1e-3, (lf, e_cell, e_norm)


def test_not_positive_definite_systems_are_flagged_and_zeroed():
    spec = synth.CPISpec(1, 4, 4, 12, 2, 4, 2, cnr_db=None, seed=51)   # D=2, 4 x 3 systems
    d = oracle.Dims(*spec.dims())
    rng = np.random.default_rng(5)
    cov = np.zeros((4, 3, 2, 2), np.complex128)
    for k in range(4):
        for b in range(3):
            M = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
            cov[k, b] = M @ M.conj().T + np.eye(2)
    cov[1, 2] = np.diag([1.0, -5.0])                 # indefinite, negative trace
    cov[3, 0, 0, 0] = np.nan                         # non-finite input
    ref, status, nf = oracle.weights(d, cov)
    assert nf == 2
    plan = _plan(spec)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    code, failed = plan.status()
    assert code == stap.STAP_ERR_NOT_POSDEF and failed == 2
    assert np.all(wts[1, 2] == 0) and np.all(wts[3, 0] == 0)
    good = status == 0
    err = np.linalg.norm(wts[good] - ref[good], axis=-1) / np.linalg.norm(ref[good], axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2)
    assert plan.status() == (stap.STAP_OK, 0)        # cleared by the previous read


def test_standard_workload_full_size_parity_and_launch_configuration():
    """The benchmark workload at full size, through the same run_cpi call the
    benchmark times, against the oracle on every cell."""
    spec = synth.standard_cpi()
    d = oracle.Dims(*spec.dims())
    cube = _cube(spec)
    res = oracle.run(d, cube, keep=True)
    plan = _plan(spec)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    e_cell, e_norm = power_errors(out, res["out"])
    print(f"standard workload: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= 1e-5 and e_cell <= PLAIN_CELL_BAR


@pytest.mark.parametrize("spec", [synth.small_cpi(), synth.standard_cpi(), EDGE_SPECS[2], EDGE_SPECS[3],
                                  EDGE_SPECS[8], EDGE_SPECS[9]],
                         ids=["small", "standard", "edge2", "edge3", "edge8", "edge9"])
def test_generic_and_separable_solves_agree(spec):
    """The default steering table is solved on the C basis vectors; the same
    table given explicitly takes the generic path (one solve per steering
    vector).  Both must match the oracle's weights."""
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, _ = oracle.weights(d, cov)
    covd = _dev(cov, torch.complex128)
    sep = _plan(spec)
    gen = _plan(spec)
    gen.set_steering(oracle.default_steering(d))
    for plan in (sep, gen):
        wts = to_np(plan.solve_weights(covd))
        err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
        assert np.max(err) <= 2 * EPS32 * np.sqrt(2), np.max(err)


@pytest.mark.parametrize("separable", [True, False], ids=["sep", "explicit"])
@pytest.mark.parametrize("lr", [8, 16, 32])
def test_per_cta_solve_with_idle_lane_groups(lr, separable):
    """One system per CTA with LR lanes per right-hand side: D = 40 and S = 5
    leave a warp holding both a live and an idle lane group (LR = 8, 16), so
    the normalisation's group-wide sum runs in every group and only live
    groups store.  Weights must match the oracle at every LR."""
    spec = synth.CPISpec(10, 16, 16, 128, 4, 64, 5, cnr_db=35.0, seed=26)   # D = 40, S = 5
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, nf = oracle.weights(d, cov)
    assert nf == 0
    plan = _plan(spec)
    if not separable:
        plan.set_steering(oracle.default_steering(d))
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[4] = lr
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    assert plan.status() == (stap.STAP_OK, 0)
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2), np.max(err)
    plan.close()


def test_pivot_reciprocal_is_within_one_ulp_of_ieee_division():
    """The FP64 factorisation's pivot reciprocal (Newton-Raphson steps from the
    hardware's approximate reciprocal) against IEEE division, over normal
    positive doubles of every magnitude whose reciprocal is normal too."""
    rng = np.random.default_rng(71)
    x = np.concatenate([2.0 ** rng.uniform(-1000.0, 1000.0, 200000), rng.uniform(1e-3, 1e3, 200000),
                        [1.0, 2.0, 3.0, 0.1, 1e-300, 1e300, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0)]])
    got = stap.stap_test_pivot_reciprocal(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    ulps = np.abs(got - ref) / np.spacing(ref)
    print(f"pivot reciprocal: max {np.max(ulps):.2f} ulp, {np.mean(ulps > 0):.3%} not correctly rounded")
    assert np.max(ulps) <= 1.0


# D > 64 systems for the one-system-per-CTA kernels: an odd D (the two-column
# factorisation rounds end with a single column) whose steering count leaves
# idle lane groups and is below 2 C (the refinement option then solves the S
# vectors directly), and D = 128 with S = 2 C (the refinement option parks the
# basis solutions in the weight rows).
LARGE_SPECS = {
    "D75": synth.CPISpec(25, 16, 16, 192, 3, 96, 7, cnr_db=35.0, seed=61),
    "D128": synth.CPISpec(32, 16, 16, 512, 4, 256, 64, cnr_db=40.0, seed=62),
}


@pytest.mark.parametrize("separable", [True, False], ids=["sep", "explicit"])
@pytest.mark.parametrize("variant", [(16, 0), (32, 0), (32, 16)], ids=["lr16", "lr32", "lr32x16warps"])
@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("name", list(LARGE_SPECS))
def test_large_per_cta_solve_variants(name, refine, variant, separable):
    """Every launch shape of the D > 64 FP64 solve (16 lanes x 8 rows, 32 x 4
    with 8 or 16 warps) against the oracle's weights."""
    spec = LARGE_SPECS[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, nf = oracle.weights(d, cov)
    assert nf == 0
    plan = _plan(spec, refine_steps=refine)
    if not separable:
        plan.set_steering(oracle.default_steering(d))
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[4], choices[3] = variant
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    assert plan.status() == (stap.STAP_OK, 0)
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2), np.max(err)
    plan.close()


@pytest.mark.parametrize("lr", [16, 32])
@pytest.mark.parametrize("name", list(LARGE_SPECS))
def test_large_refinement_solve_variants(name, lr):
    """The refinement option's D > 64 form (FP32 factor in shared memory with
    the double-float Rl) at both launch shapes, 2 steps."""
    spec = LARGE_SPECS[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, nf = oracle.weights(d, cov)
    assert nf == 0
    plan = _plan(spec, refine_steps=2, solver=stap.STAP_SOLVE_MIXED_IR)
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[4] = lr
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    assert plan.status() == (stap.STAP_OK, 0)
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert np.max(err) <= 4 * EPS32, np.max(err)
    plan.close()


# Snapshot lengths with a register-resident solve kernel (D = 8, 12, 16), each
# with a steering count that leaves idle lanes in the last pass.
REG_SPECS = {
    "D8": synth.CPISpec(4, 16, 32, 128, 2, 32, 6, cnr_db=35.0, seed=21),
    "D12": synth.CPISpec(3, 24, 32, 96, 4, 32, 5, cnr_db=40.0, seed=22),
    "D16": synth.CPISpec(8, 16, 16, 128, 2, 64, 12, cnr_db=40.0, seed=23),
}


SMALL_SPECS = dict(REG_SPECS)
SMALL_SPECS.update({
    "D6": synth.CPISpec(3, 20, 32, 96, 2, 32, 5, cnr_db=30.0, seed=11),
    "D24": synth.CPISpec(8, 16, 32, 128, 3, 64, 9, cnr_db=35.0, seed=25),
})


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("separable", [True, False], ids=["sep", "explicit"])
@pytest.mark.parametrize("name", list(SMALL_SPECS))
def test_register_and_shared_memory_solves_match_the_oracle(name, separable, refine):
    """The small-system solve kernels (tuning choice 8: 1 register-resident
    LDL^H where D = 8, 12, 16, 2 shared-memory Cholesky teams, 3 one system per
    CTA) on the default separable steering and on the same table given
    explicitly (one solve per steering vector)."""
    spec = SMALL_SPECS[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, nf = oracle.weights(d, cov)
    assert nf == 0
    covd = _dev(cov, torch.complex128)
    out = {}
    for kind in (1, 2, 3):
        plan = _plan(spec, refine_steps=refine)
        if not separable:
            plan.set_steering(oracle.default_steering(d))
        choices = stap.stap_plan_get_tuning(plan.handle, 0)
        choices[7] = kind
        stap.stap_plan_set_tuning(plan.handle, 0, choices)
        wts = to_np(plan.solve_weights(covd))
        assert plan.status() == (stap.STAP_OK, 0)
        err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
        assert np.max(err) <= 2 * EPS32 * np.sqrt(2), (kind, np.max(err))
        out[kind] = wts
        plan.close()
    for kind in (1, 3):
        diff = np.linalg.norm(out[kind] - out[2], axis=-1) / np.linalg.norm(out[2], axis=-1)
        assert np.max(diff) <= 4 * EPS32, (kind, np.max(diff))


@pytest.mark.parametrize("kind", [1, 2, 3], ids=["register", "shared", "per_cta"])
def test_not_positive_definite_flagged_by_both_small_solves(kind):
    spec = synth.CPISpec(4, 4, 4, 12, 2, 4, 3, cnr_db=None, seed=52)   # D = 8, 4 x 3 systems
    d = oracle.Dims(*spec.dims())
    rng = np.random.default_rng(6)
    cov = np.zeros((4, 3, 8, 8), np.complex128)
    for k in range(4):
        for b in range(3):
            M = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
            cov[k, b] = M @ M.conj().T + np.eye(8)
    cov[0, 1] = -np.eye(8)                           # indefinite, negative trace
    cov[2, 2, 5, 3] = np.inf                         # non-finite entry below the diagonal
    cov[2, 2, 3, 5] = np.inf
    ref, status, nf = oracle.weights(d, cov)
    assert nf == 2
    plan = _plan(spec)
    choices = stap.stap_plan_get_tuning(plan.handle, 0)
    choices[7] = kind
    stap.stap_plan_set_tuning(plan.handle, 0, choices)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    code, failed = plan.status()
    assert code == stap.STAP_ERR_NOT_POSDEF and failed == 2
    assert np.all(wts[0, 1] == 0) and np.all(wts[2, 2] == 0)
    good = status == 0
    err = np.linalg.norm(wts[good] - ref[good], axis=-1) / np.linalg.norm(ref[good], axis=-1)
    assert np.max(err) <= 2 * EPS32 * np.sqrt(2)


# ---- mixed-precision iterative refinement (STAP_SOLVE_MIXED_IR) ----
# Each refinement step shrinks the FP32 solve's error by about cond(Rl) 2^-24
# (cond ~ 1e3 D with the default load): after two steps the weights are at
# their complex64 rounding, like the FP64 solve's; one step leaves about
# (cond 2^-24)^2.

MIR_SPECS = dict(REG_SPECS)
MIR_SPECS.update({
    "D6": synth.CPISpec(3, 20, 32, 96, 2, 32, 5, cnr_db=30.0, seed=11),       # one system per CTA
    "D24": synth.CPISpec(8, 16, 32, 128, 3, 64, 9, cnr_db=35.0, seed=25),
    "D33": synth.CPISpec(11, 16, 16, 96, 3, 48, 7, cnr_db=35.0, seed=24),     # odd D, S % 8 != 0
    "D64": synth.CPISpec(16, 32, 64, 256, 4, 128, 8, cnr_db=40.0, seed=14),
    "D100": EDGE_SPECS[9],                                                      # FP32 factor,
    "D128": EDGE_SPECS[8],                                                      # FP64 residuals
})


@pytest.mark.parametrize("refine", [1, 2, 3])
@pytest.mark.parametrize("separable", [True, False], ids=["sep", "explicit"])
@pytest.mark.parametrize("name", list(MIR_SPECS))
def test_mixed_refinement_weights_match_the_oracle(name, separable, refine):
    spec = MIR_SPECS[name]
    d = oracle.Dims(*spec.dims())
    cov = oracle.covariance(d, oracle.doppler(d, _cube(spec)))
    ref, _, nf = oracle.weights(d, cov)
    assert nf == 0
    plan = _plan(spec, refine_steps=refine, solver=stap.STAP_SOLVE_MIXED_IR)
    if not separable:
        plan.set_steering(oracle.default_steering(d))
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    assert plan.status() == (stap.STAP_OK, 0)
    err = np.linalg.norm(wts - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    print(f"{name} refine={refine}: max weight error {np.max(err):.3e}")
    bar = 1e-4 if refine == 1 else 4 * EPS32
    assert np.max(err) <= bar, np.max(err)
    plan.close()


@pytest.mark.parametrize("spec", [synth.small_cpi(), synth.standard_cpi(), MIR_SPECS["D64"],
                                  MIR_SPECS["D128"]], ids=["small", "standard", "D64", "D128"])
def test_mixed_refinement_end_to_end_meets_the_plain_bar(spec):
    d = oracle.Dims(*spec.dims())
    cube = _cube(spec)
    ref = oracle.run(d, cube)["out"]
    plan = _plan(spec, refine_steps=2, solver=stap.STAP_SOLVE_MIXED_IR)
    out = to_np(plan.run_cpi(_dev(cube, torch.complex64)))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    print(f"{spec.dims()} mixed refinement: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    g = growth(spec)
    assert e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g


def test_mixed_refinement_flags_breakdown():
    spec = synth.CPISpec(4, 4, 4, 12, 2, 4, 3, cnr_db=None, seed=52)   # D = 8, 4 x 3 systems
    d = oracle.Dims(*spec.dims())
    rng = np.random.default_rng(6)
    cov = np.zeros((4, 3, 8, 8), np.complex128)
    for k in range(4):
        for b in range(3):
            M = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
            cov[k, b] = M @ M.conj().T + np.eye(8)
    cov[0, 1] = -np.eye(8)
    cov[2, 2, 0, 0] = np.nan
    ref, status, nf = oracle.weights(d, cov)
    assert nf == 2
    plan = _plan(spec, refine_steps=2, solver=stap.STAP_SOLVE_MIXED_IR)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    code, failed = plan.status()
    assert code == stap.STAP_ERR_NOT_POSDEF and failed == 2
    assert np.all(wts[0, 1] == 0) and np.all(wts[2, 2] == 0)
    good = status == 0
    err = np.linalg.norm(wts[good] - ref[good], axis=-1) / np.linalg.norm(ref[good], axis=-1)
    assert np.max(err) <= 4 * EPS32


def test_large_mixed_refinement_flags_breakdown():
    spec = synth.CPISpec(16, 4, 4, 12, 3, 4, 5, cnr_db=None, seed=53)   # D = 48, 4 x 3 systems
    d = oracle.Dims(*spec.dims())
    rng = np.random.default_rng(7)
    cov = np.zeros((4, 3, 48, 48), np.complex128)
    for k in range(4):
        for b in range(3):
            M = rng.standard_normal((48, 48)) + 1j * rng.standard_normal((48, 48))
            cov[k, b] = M @ M.conj().T + np.eye(48)
    cov[1, 0] = -np.eye(48)
    cov[3, 2, 20, 20] = np.inf
    ref, status, nf = oracle.weights(d, cov)
    assert nf == 2
    plan = _plan(spec, refine_steps=2, solver=stap.STAP_SOLVE_MIXED_IR)
    wts = to_np(plan.solve_weights(_dev(cov, torch.complex128)))
    code, failed = plan.status()
    assert code == stap.STAP_ERR_NOT_POSDEF and failed == 2
    assert np.all(wts[1, 0] == 0) and np.all(wts[3, 2] == 0)
    good = status == 0
    err = np.linalg.norm(wts[good] - ref[good], axis=-1) / np.linalg.norm(ref[good], axis=-1)
    assert np.max(err) <= 4 * EPS32
