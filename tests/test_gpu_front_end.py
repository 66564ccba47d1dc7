"""Reduced-DOF front end (stap_plan_set_front_end / stap_reduce_channels):
N element channels combined into the plan's C channels by W[C][N], then the
unchanged chain with the reduced steering.  Parity with the oracle's
oracle_reduce_channels / oracle_reduced_steering."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2203_06233_gb300 import stap, synth

from _parity import EPS32, PLAIN_CELL_BAR, power_errors, to_np

pytestmark = pytest.mark.gpu

# element cube of N = 32 elements; C = 4 subarrays of 8
ELEM = synth.CPISpec(32, 32, 32, 256, 3, 32, 4, cnr_db=30.0,
                     targets=(synth.Target(128, 24, 2, 10.0, 0.3),), seed=61)


def _reduced_spec(elem, C):
    return dataclasses.replace(elem, n_chan=C)


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dtype)


@pytest.mark.parametrize("N,C,P,K,R,B", [(77, 3, 16, 16, 64, 16),     # P R even: bulk-copy kernel
                                          (77, 6, 5, 8, 63, 9),       # P R odd: register kernel
                                          (1000, 4, 4, 4, 1030, 10)],  # ragged last tile
                         ids=["bulk", "odd", "ragged"])
def test_reduce_channels_matches_the_oracle_within_the_fp32_sum_bound(N, C, P, K, R, B):
    rng = np.random.default_rng(7)
    spec = synth.CPISpec(C, P, K, R, 2, B, 4, cnr_db=None, seed=62)
    W = rng.standard_normal((C, N)) + 1j * rng.standard_normal((C, N))
    x = (rng.standard_normal((N, P, R)) + 1j * rng.standard_normal((N, P, R))).astype(np.complex64)
    ref = oracle.reduce_channels(W, x)
    plan = stap.Plan(spec.dims(), front_end=W)
    y = to_np(plan.reduce_channels(_dev(x)))
    # FP32: W rounded once, each product and each addition of the 32-element
    # block sums and of the block totals rounded once
    steps = 2 * min(N, 32) + math.ceil(N / 32) + 4
    mag = np.einsum("cn,npr->cpr", np.abs(W), np.abs(x.astype(np.complex128)))
    bound = steps * EPS32 * 2.0 * mag
    assert np.all(np.abs(y - ref) <= bound), float(np.max(np.abs(y - ref) / bound))
    plan.close()


def test_identity_front_end_is_the_plain_path_bit_for_bit():
    spec = synth.small_cpi()
    x = torch.from_numpy(synth.make_cube(spec)).cuda()
    plain = stap.Plan(spec.dims())
    fe = stap.Plan(spec.dims(), front_end=np.eye(spec.n_chan, dtype=np.complex128))
    y = fe.reduce_channels(x)
    assert torch.equal(y, x)
    assert torch.equal(fe.run_cpi(y), plain.run_cpi(x))
    plain.close()
    fe.close()


@pytest.mark.parametrize("C", [4, 8])
def test_subarray_front_end_end_to_end_matches_the_oracle(C):
    spec = _reduced_spec(ELEM, C)
    d = oracle.Dims(*spec.dims())
    W = oracle.subarray_weights(ELEM.n_chan, C)
    x = synth.make_cube(ELEM)
    y_ref = oracle.reduce_channels(W, x)
    ref = oracle.run(d, y_ref, steer=oracle.reduced_steering(d, W))["out"]
    plan = stap.Plan(spec.dims(), front_end=W)
    out = to_np(plan.run_cpi(plan.reduce_channels(_dev(x))))
    assert plan.status() == (stap.STAP_OK, 0)
    e_cell, e_norm = power_errors(out, ref)
    g = max(1.0, (spec.D + 2) / 14.0)
    print(f"C{C}: max-cell/floor={e_cell:.3e} normwise={e_norm:.3e}")
    assert e_norm <= 1e-5 * g and e_cell <= PLAIN_CELL_BAR * g
    assert int(np.argmax(out[2, 24])) == 128           # the target through the subarrays
    plan.close()


def test_streamed_element_cubes_equal_the_device_path_with_one_chunk():
    C = 4
    spec = _reduced_spec(ELEM, C)
    W = oracle.subarray_weights(ELEM.n_chan, C)
    cubes = [torch.from_numpy(synth.make_cube(dataclasses.replace(ELEM, seed=70 + i))) for i in range(3)]
    plan = stap.Plan(spec.dims(), front_end=W, front_end_chunk=ELEM.n_chan)   # one chunk
    ref = [plan.run_cpi(plan.reduce_channels(c.cuda())).cpu() for c in cubes]
    outs = plan.run_stream([c.pin_memory() for c in cubes])
    torch.cuda.current_stream().synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    assert plan.status() == (stap.STAP_OK, 0)
    plan.close()


def test_streamed_element_cubes_in_chunks_match_the_oracle():
    """Chunks of 5 of the 32 elements (7 copies and reductions per cube): the
    streamed outputs meet the end-to-end bar against the oracle."""
    C = 4
    spec = _reduced_spec(ELEM, C)
    d = oracle.Dims(*spec.dims())
    W = oracle.subarray_weights(ELEM.n_chan, C)
    specs = [dataclasses.replace(ELEM, seed=80 + i) for i in range(3)]
    cubes = [synth.make_cube(s) for s in specs]
    plan = stap.Plan(spec.dims(), front_end=W, front_end_chunk=5)
    outs = plan.run_stream([torch.from_numpy(c).pin_memory() for c in cubes])
    torch.cuda.current_stream().synchronize()
    assert plan.status() == (stap.STAP_OK, 0)
    steer = oracle.reduced_steering(d, W)
    for o, x in zip(outs, cubes):
        ref = oracle.run(d, oracle.reduce_channels(W, x), steer=steer)["out"]
        e_cell, e_norm = power_errors(o.numpy(), ref)
        assert e_norm <= 1e-5 and e_cell <= PLAIN_CELL_BAR, (e_norm, e_cell)
    plan.close()


def test_autotune_keeps_the_front_end_table(tmp_path):
    """The slab search evicts the L2 by writing the intermediates; the W table
    stored after them must survive it."""
    spec = _reduced_spec(ELEM, 4)
    W = oracle.subarray_weights(ELEM.n_chan, 4)
    x = _dev(synth.make_cube(ELEM))
    plan = stap.Plan(spec.dims(), front_end=W)
    y = plan.reduce_channels(x).clone()
    out = torch.empty(plan.shapes()["out"], dtype=torch.float32, device="cuda")
    plan.autotune(y, out, cache_path=str(tmp_path / "tune.json"), force=True)
    assert torch.equal(plan.reduce_channels(x), y)
    plan.close()
