"""Parity of the mixed-precision paths with the FP64 oracle: the covariance
and the apply on the tensor cores (tcgen05) as split products with FP32
accumulation, in each of the three arithmetics (STAP_PREC_TF32X3,
STAP_PREC_BF16X3, STAP_PREC_FP16_SCALED); the FP64 solve is unchanged.

Per-product error of the split arithmetics, relative to the product's own
size (TF32X3: about 3 x 2^-22; BF16X3: about 3 x 2^-25) or, for the
per-block-scaled FP16, to the block's largest magnitudes (the pieces hold 22
bits of the scaled values, so a value's error is at most 2^-22 of its
block's largest magnitude, and a product of two such values is off by at
most about 3 x 2^-22 of the product of the two block maxima).

Tolerances:
- covariance per system, relative Frobenius: <= max(1e-5, 2 B u) (u = 2^-24:
  the split products plus FP32 accumulation of B terms) for TF32X3 and
  BF16X3; FP16_SCALED adds 8 D 2^-22 m^2 / ||R||_F with m the system's
  largest magnitude (two real products per component of an entry, each off
  by at most 3 x 2^-22 m^2, rounded up; D^2 entries in the Frobenius norm);
- apply, every cell within 2|y| g + g^2 + 2 u P with g = (2 D + 8) u
  sum |w||x| (FP32 accumulation of 2 D real products, each within 3 u of its
  own size for TF32X3/BF16X3), plus for FP16_SCALED 10 D 2^-22 wmax xmax
  (2 D real products per component, each off by at most 3 x 2^-22 wmax xmax
  with xmax the tile's largest snapshot value and wmax the weight vector's
  largest value; sqrt(2) for the complex magnitude, rounded up);
- whole path normwise <= 1e-3 (the mixed bar) and every cell within
  mixed_cell_bar of max(P_ref, median P_ref) (the first-order effect of the
  covariance error, 2 x 2^-21 (D/lf + 1))."""
import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import (EDGE_SPECS, EPS32, MIXED_NORM_BAR, MIXED_PRECISIONS, mixed_cell_bar,
                     power_errors, to_np)

pytestmark = pytest.mark.gpu

SPECS = [synth.small_cpi(), synth.standard_cpi()] + EDGE_SPECS
IDS = ["small", "standard"] + [f"edge{i}" for i in range(len(EDGE_SPECS))]
PRECS = [p for _, p in MIXED_PRECISIONS]
PIDS = [n for n, _ in MIXED_PRECISIONS]
EPS_F16S = 2.0 ** -22


def growth(spec):
    return max(1.0, (spec.D + 2) / 14.0)


def _plan(spec, prec):
    return stap.Plan(spec.dims(), precision=prec)


@pytest.mark.parametrize("prec", PRECS, ids=PIDS)
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_mixed_covariance_parity(spec, prec):
    _check_covariance(spec, prec)


# Snapshot lengths whose tensor-core tile is wider than its systems' rows:
# D8 = D rounded up to 8 is 40 or 56, so the accumulator (G D8 rounded up to
# 16 columns) also takes rows of the Xi block or zero rows as columns that
# the epilogue must ignore; D = 24 packs two systems per tile, and D = 72
# runs the four-accumulator form with 80 columns per accumulator.
WIDTH_SPECS = [synth.CPISpec(10, 16, 16, 256, 4, 64, 4, cnr_db=30.0, seed=31),   # D = 40
               synth.CPISpec(12, 16, 16, 256, 3, 64, 4, cnr_db=30.0, seed=32),   # D = 36
               synth.CPISpec(14, 16, 16, 256, 4, 64, 4, cnr_db=30.0, seed=33),   # D = 56
               synth.CPISpec(8, 16, 16, 256, 3, 64, 4, cnr_db=30.0, seed=34),    # D = 24
               synth.CPISpec(18, 16, 16, 256, 4, 128, 4, cnr_db=30.0, seed=35)]  # D = 72


@pytest.mark.parametrize("prec", PRECS, ids=PIDS)
@pytest.mark.parametrize("spec", WIDTH_SPECS, ids=[f"D{s.D}" for s in WIDTH_SPECS])
def test_mixed_covariance_tile_widths(spec, prec):
    _check_covariance(spec, prec)


def _check_covariance(spec, prec):
    from _parity import gather
    d = oracle.Dims(*spec.dims())
    dop64 = oracle.doppler(d, synth.make_cube(spec)).astype(np.complex64)
    ref = oracle.covariance(d, dop64)
    plan = _plan(spec, prec)
    cov = to_np(plan.covariance(torch.from_numpy(dop64).cuda()))
    assert plan.status() == (stap.STAP_OK, 0)
    np.testing.assert_array_equal(cov, np.conj(np.swapaxes(cov, -1, -2)))
    num = np.linalg.norm((cov - ref).reshape(spec.n_dop, spec.NB, -1), axis=-1)
    den = np.linalg.norm(ref.reshape(spec.n_dop, spec.NB, -1), axis=-1)
    tol = np.full(den.shape, max(1e-5, 2 * spec.training_block * EPS32))
    if prec == stap.STAP_PREC_FP16_SCALED:
        x = gather(dop64.astype(np.complex128), spec.tdof)                    # [K][R][D]
        comp = np.maximum(np.abs(x.real), np.abs(x.imag))
        m = comp.reshape(spec.n_dop, spec.NB, -1).max(axis=-1)                # [K][NB]
        tol = tol + 8 * spec.D * EPS_F16S * m * m / den
    rel = num / den
    print(f"{spec.dims()} prec {prec}: max per-system rel err {np.max(rel):.3e} "
          f"(tol min {np.min(tol):.1e})")
    assert np.all(rel <= tol)


@pytest.mark.parametrize("prec", PRECS, ids=PIDS)
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_mixed_run_cpi_end_to_end(spec, prec):
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    ref = oracle.run(d, cube)["out"]
    plan = _plan(spec, prec)
    out = to_np(plan.run_cpi(torch.from_numpy(cube).cuda()))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    print(f"{spec.dims()}: mixed prec {prec} max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= MIXED_NORM_BAR and e_cell <= mixed_cell_bar(spec), (e_cell, e_norm)


@pytest.mark.parametrize("prec", PRECS, ids=PIDS)
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_mixed_apply_parity(spec, prec):
    """Tensor-core apply (where the tile shape allows it; the FP32 apply
    otherwise) against the oracle on the same complex64 inputs: every cell
    within the bound of the module docstring."""
    from _parity import gather
    d = oracle.Dims(*spec.dims())
    dop = oracle.doppler(d, synth.make_cube(spec))
    w, _, _ = oracle.weights(d, oracle.covariance(d, dop))
    dop64, w64 = dop.astype(np.complex64), w.astype(np.complex64)
    ref = oracle.apply(d, dop64, w64)
    plan = _plan(spec, prec)
    out = to_np(plan.apply(torch.from_numpy(dop64).cuda(), torch.from_numpy(w64).cuda()))
    assert plan.status() == (stap.STAP_OK, 0)
    x = gather(dop64.astype(np.complex128), spec.tdof)                        # [K][R][D]
    wb = np.repeat(w64.astype(np.complex128), spec.training_block, axis=1)     # [K][R][S][D]
    y = np.einsum("krsd,krd->skr", wb.conj(), x)
    mag = np.einsum("krsd,krd->skr", np.abs(wb), np.abs(x))
    g = (2 * spec.D + 8) * EPS32 * mag
    if prec == stap.STAP_PREC_FP16_SCALED:
        K, R = spec.n_dop, spec.n_range
        comp = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=-1)         # [K][R]
        nt = (R + 127) // 128
        pad = np.zeros((K, nt * 128))
        pad[:, :R] = comp
        xmax = np.repeat(pad.reshape(K, nt, 128).max(axis=-1), 128, axis=1)[:, :R]   # [K][R]
        wmax = np.maximum(np.abs(wb.real), np.abs(wb.imag)).max(axis=-1)       # [K][R][S]
        g = g + 10 * spec.D * EPS_F16S * np.transpose(wmax, (2, 0, 1)) * xmax[None]
    bound = 2 * np.abs(y) * g + g * g + 2 * EPS32 * np.abs(y) ** 2
    viol = np.abs(out - ref) > bound
    assert not viol.any(), (int(viol.sum()), float(np.max(np.abs(out - ref) - bound)))


@pytest.mark.parametrize("step", ["covariance", "apply"])
def test_pipeline_wait_limit_reports_timeout_and_next_call_runs_clean(step):
    """With a pipeline wait limit of 0 polls every tensor-core CTA gives up at
    its first wait on an MMA commit: it records the timeout, drains the MMAs it
    issued (with the default limit), frees its TMEM and exits.  The host reads
    STAP_ERR_TIMEOUT, the status is then clear, and with the default limit
    restored the same call gives the result of a fresh plan.  Nothing here
    waits on something that never happens: the MMAs complete normally, the
    waits just stop looking early."""
    spec = synth.CPISpec(16, 32, 64, 256, 4, 128, 8, cnr_db=40.0, seed=14)   # D = 64
    d = oracle.Dims(*spec.dims())
    dop = oracle.doppler(d, synth.make_cube(spec)).astype(np.complex64)
    w, _, _ = oracle.weights(d, oracle.covariance(d, dop))
    dop_d = torch.from_numpy(dop).cuda()
    w_d = torch.from_numpy(w.astype(np.complex64)).cuda()
    fresh = _plan(spec, stap.STAP_PREC_TF32X3)
    want = fresh.covariance(dop_d) if step == "covariance" else fresh.apply(dop_d, w_d)
    assert fresh.status() == (stap.STAP_OK, 0)
    plan = _plan(spec, stap.STAP_PREC_TF32X3)
    plan.set_wait_limit(0)
    plan.covariance(dop_d) if step == "covariance" else plan.apply(dop_d, w_d)
    assert plan.status()[0] == stap.STAP_ERR_TIMEOUT
    assert plan.status() == (stap.STAP_OK, 0)          # read and cleared
    plan.set_wait_limit()                               # the default limit again
    got = plan.covariance(dop_d) if step == "covariance" else plan.apply(dop_d, w_d)
    assert plan.status() == (stap.STAP_OK, 0)
    assert torch.equal(got, want)
    with pytest.raises(stap.StapError):
        plan.set_wait_limit(-1)
