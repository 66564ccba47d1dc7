"""Host-side tests of the C ABI: the library loads without a GPU, exports every
symbol ``include/stap.h`` declares, and validates shapes, options, pointers and
workspace sizes before touching CUDA (none of these calls launches anything)."""
import ctypes
import os
import re

import pytest

from paper_2203_06233_gb300 import stap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

GOOD = (4, 128, 256, 4096, 3, 64, 16)


def _declared():
    src = open(os.path.join(ROOT, "include", "stap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stap_[a-z_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    L = stap.lib()
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(L, name), f"{name} declared in stap.h but not exported"
    assert set(declared) == set(stap.EXPORTED)
    assert stap.stap_abi_version() == 5


def _create(dims, opts=None):
    L = stap.lib()
    arr = (stap.stap_dims * 1)(stap.stap_dims(*dims))
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    code = L.stap_plan_create(arr, 1, ctypes.byref(opts) if opts else None, None, ctypes.byref(h),
                              ctypes.byref(ws))
    return code, h, ws.value


def test_plan_create_default_options_and_workspace_layout():
    o = stap.stap_options_default()
    assert o.load_factor == 1e-3 and o.refine_steps == 1 and o.precision == 0
    code, h, ws = _create(GOOD)
    assert code == stap.STAP_OK and h.value
    step, run = stap.stap_plan_workspace_sizes(h)
    C, P, K, R, T, B, S = GOOD
    D, NB = C * T, R // B
    inter = C * K * R * 8 + K * NB * D * D * 16 + K * NB * S * D * 8
    assert run == ws
    # three 256-byte aligned regions plus the alignment slack of 8 range slabs
    assert run - step >= inter and run - step < inter + 4 * 256 + 2 * 8 * 256
    assert step < 64 * 1024                                 # status + window + twiddles + steering
    stap.stap_plan_destroy(h)


@pytest.mark.parametrize("dims,code", [
    ((0, 128, 256, 4096, 3, 64, 16), stap.STAP_ERR_SHAPE),      # no channels
    ((4, 128, 64, 4096, 3, 64, 16), stap.STAP_ERR_SHAPE),       # K < P
    ((4, 128, 256, 4000, 3, 64, 16), stap.STAP_ERR_SHAPE),      # R not a multiple of B
    ((4, 8, 8, 64, 9, 8, 4), stap.STAP_ERR_SHAPE),              # T > K
    ((4, 128, 256, 4096, 3, 64, 0), stap.STAP_ERR_SHAPE),       # no steering vectors
    ((4, 128, 192, 4096, 3, 64, 16), stap.STAP_ERR_UNSUPPORTED),  # K not a power of two
    ((4, 128, 2048, 4096, 3, 64, 16), stap.STAP_ERR_UNSUPPORTED),  # K > 1024
    ((65, 16, 16, 64, 2, 8, 4), stap.STAP_ERR_UNSUPPORTED),     # D = 130 > 128
])
def test_plan_create_rejects_bad_shapes(dims, code):
    got, h, _ = _create(dims)
    assert got == code and not h.value


@pytest.mark.parametrize("lf,refine,prec,solver,code", [
    (-1.0, 1, 0, 0, stap.STAP_ERR_INVALID_ARG),
    (float("nan"), 1, 0, 0, stap.STAP_ERR_INVALID_ARG),
    (1e-3, -1, 0, 0, stap.STAP_ERR_INVALID_ARG),
    (1e-3, 5, 0, 0, stap.STAP_ERR_INVALID_ARG),
    (1e-3, 1, 7, 0, stap.STAP_ERR_UNSUPPORTED),
    (1e-3, 1, 4, 0, stap.STAP_ERR_UNSUPPORTED),
    (1e-3, 1, 1, 0, stap.STAP_OK),             # BF16X3
    (1e-3, 1, 2, 0, stap.STAP_OK),             # TF32X3
    (1e-3, 1, 3, 0, stap.STAP_OK),             # FP16_SCALED
    (0.0, 0, 0, 0, stap.STAP_OK),
    (1e-3, 2, 0, 1, stap.STAP_OK),             # mixed-precision refinement, D = 12
    (1e-3, 2, 2, 1, stap.STAP_OK),
    (1e-3, 2, 0, 2, stap.STAP_ERR_UNSUPPORTED),
])
def test_plan_create_checks_options(lf, refine, prec, solver, code):
    got, h, _ = _create(GOOD, stap.stap_options(lf, refine, prec, solver))
    assert got == code
    if h.value:
        stap.stap_plan_destroy(h)


def test_training_option_values_and_block_count():
    o = stap.stap_options_default()
    assert o.training == stap.STAP_TRAIN_OWN_BLOCK
    assert o.train_guard == 0 and o.train_half == 1
    W = stap.STAP_TRAIN_WINDOW
    for training, dims, guard, half, code in [
            (1, GOOD, 0, 0, stap.STAP_OK),
            (3, GOOD, 0, 1, stap.STAP_ERR_INVALID_ARG),
            (-1, GOOD, 0, 1, stap.STAP_ERR_INVALID_ARG),
            (1, (4, 16, 32, 64, 2, 64, 4), 0, 1, stap.STAP_ERR_SHAPE),           # NB = 1
            (1, (4, 16, 32, 128, 2, 64, 4), 0, 1, stap.STAP_OK),                 # NB = 2
            (W, GOOD, 2, 16, stap.STAP_OK),
            (W, GOOD, 0, 0, stap.STAP_ERR_INVALID_ARG),                          # half < 1
            (W, GOOD, -1, 1, stap.STAP_ERR_INVALID_ARG),
            (W, (4, 16, 32, 128, 2, 1, 4), 63, 4, stap.STAP_OK),                 # NB = 128 = 2 g + 2
            (W, (4, 16, 32, 128, 2, 1, 4), 64, 4, stap.STAP_ERR_SHAPE)]:         # NB < 2 g + 2
        got, h, _ = _create(dims, stap.stap_options(1e-3, 1, 0, 0, training, 0, guard, half))
        assert got == code, (training, dims, guard, half)
        if h.value:
            stap.stap_plan_destroy(h)


def test_training_workspace_holds_the_training_matrices():
    C, P, K, R, T, B, S = GOOD
    D, NB = C * T, R // B
    _, h0, ws0 = _create(GOOD)
    _, h1, ws1 = _create(GOOD, stap.stap_options(1e-3, 1, 0, 0, 1))
    _, h2, ws2 = _create(GOOD, stap.stap_options(1e-3, 1, 0, 0, stap.STAP_TRAIN_WINDOW, 0, 1, 4))
    assert ws1 - ws0 >= K * NB * D * D * 16 and ws1 - ws0 < K * NB * D * D * 16 + 512
    assert ws2 == ws1
    for h in (h0, h1, h2):
        stap.stap_plan_destroy(h)


def test_snapshot_option_values_and_pulse_limit():
    o = stap.stap_options_default()
    assert o.snapshots == stap.STAP_SNAP_ADJACENT_BINS
    for snaps, dims, code in [(1, GOOD, stap.STAP_OK),
                              (2, GOOD, stap.STAP_ERR_INVALID_ARG),
                              (-1, GOOD, stap.STAP_ERR_INVALID_ARG),
                              (1, (4, 2, 32, 64, 3, 16, 4), stap.STAP_ERR_SHAPE),   # T > P
                              (0, (4, 2, 32, 64, 3, 16, 4), stap.STAP_OK),          # adjacent bins
                              (1, (4, 3, 32, 64, 3, 16, 4), stap.STAP_OK)]:         # one-pulse sub-windows
        got, h, _ = _create(dims, stap.stap_options(1e-3, 1, 0, 0, 0, snaps))
        assert got == code, (snaps, dims)
        if h.value:
            stap.stap_plan_destroy(h)


def test_staggered_workspace_holds_the_wider_doppler_cube():
    """PRI-staggered snapshots: the Doppler intermediate has C*T rows, not C."""
    C, P, K, R, T, B, S = GOOD
    _, h0, ws0 = _create(GOOD)
    _, h1, ws1 = _create(GOOD, stap.stap_options(1e-3, 1, 0, 0, 0, stap.STAP_SNAP_PRI_STAGGERED))
    extra = (T - 1) * C * K * R * 8
    assert abs((ws1 - ws0) - extra) <= 256
    stap.stap_plan_destroy(h0)
    stap.stap_plan_destroy(h1)


def test_stream_workspace_and_arguments_fail_before_cuda():
    L = stap.lib()
    C, P, K, R, T, B, S = GOOD
    code, h, ws = _create(GOOD)
    assert code == 0
    sb = ctypes.c_size_t()
    assert L.stap_plan_stream_bytes(h, ctypes.byref(sb)) == stap.STAP_OK
    cube_b, out_b = C * P * R * 8, S * K * R * 4
    assert sb.value >= ws + 2 * cube_b + 2 * out_b and sb.value <= ws + 2 * cube_b + 2 * out_b + 1024
    assert L.stap_plan_stream_bytes(h, None) == stap.STAP_ERR_INVALID_ARG
    fake = ctypes.c_void_p(0x10000)                           # never dereferenced
    arr = (ctypes.c_void_p * 1)(fake)
    nul = (ctypes.c_void_p * 1)(None)
    assert L.stap_run_stream(h, -1, arr, arr) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_run_stream(h, 1, None, arr) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_run_stream(h, 1, arr, nul) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_run_stream(h, 1, arr, arr) == stap.STAP_ERR_NO_WORKSPACE
    stap.stap_plan_destroy(h)
    # a batch plan has no streamed form
    dims2 = (stap.stap_dims * 2)(stap.stap_dims(*GOOD), stap.stap_dims(*GOOD))
    h2 = ctypes.c_void_p()
    assert L.stap_plan_create(dims2, 2, None, None, ctypes.byref(h2), None) == stap.STAP_OK
    assert L.stap_plan_stream_bytes(h2, ctypes.byref(sb)) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_run_stream(h2, 1, arr, arr) == stap.STAP_ERR_INVALID_ARG
    stap.stap_plan_destroy(h2)


def test_front_end_arguments_and_workspace_growth():
    import numpy as np
    L = stap.lib()
    C, P, K, R, T, B, S = GOOD
    N = 1000
    W = np.zeros((C, N), np.complex128)
    W[:, :4] = np.eye(C)
    Wp = W.ctypes.data_as(ctypes.c_void_p)
    code, h, ws = _create(GOOD)
    step, run = stap.stap_plan_workspace_sizes(h)
    sb0 = stap.stap_plan_stream_bytes(h)
    assert L.stap_plan_set_front_end(h, 0, Wp, 0) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_plan_set_front_end(h, N, None, 0) == stap.STAP_ERR_INVALID_ARG
    bad = W.copy()
    bad[1, 7] = np.nan
    assert L.stap_plan_set_front_end(h, N, bad.ctypes.data_as(ctypes.c_void_p), 0) == stap.STAP_ERR_INVALID_ARG
    fake = ctypes.c_void_p(0x10000)                           # never dereferenced
    assert L.stap_reduce_channels(h, fake, fake) == stap.STAP_ERR_INVALID_ARG   # no front end yet
    assert L.stap_plan_set_front_end(h, N, Wp, 0) == stap.STAP_OK
    assert L.stap_plan_set_front_end(h, N, Wp, 0) == stap.STAP_ERR_INVALID_ARG  # only once
    step1, run1 = stap.stap_plan_workspace_sizes(h)
    assert step1 == step and 0 <= run1 - run - C * N * 8 < 256
    # default chunk: 128 element rows of 4 MiB (512 MiB); the stream holds the
    # reduced cube, two chunks and two outputs beyond the run workspace
    PR8 = P * R * 8
    sb1 = stap.stap_plan_stream_bytes(h)
    expect = run1 + C * PR8 + 2 * 128 * PR8 + 2 * S * K * R * 4
    assert 0 <= sb1 - expect < 1024 and sb1 != sb0
    assert L.stap_reduce_channels(h, fake, fake) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_reduce_channels(h, ctypes.c_void_p(0x10008), fake) == stap.STAP_ERR_MISALIGNED
    stap.stap_plan_destroy(h)
    dims2 = (stap.stap_dims * 2)(stap.stap_dims(*GOOD), stap.stap_dims(*GOOD))
    h2 = ctypes.c_void_p()
    assert L.stap_plan_create(dims2, 2, None, None, ctypes.byref(h2), None) == stap.STAP_OK
    assert L.stap_plan_set_front_end(h2, N, Wp, 0) == stap.STAP_ERR_INVALID_ARG   # batch plan
    stap.stap_plan_destroy(h2)


def test_options_default_and_mixed_refinement_shape_limits():
    o = stap.stap_options_default()
    assert o.solver == stap.STAP_SOLVE_FP64
    mir = stap.stap_options(1e-3, 2, 0, stap.STAP_SOLVE_MIXED_IR)
    for dims, code in [((4, 16, 32, 256, 2, 32, 4), stap.STAP_OK),          # D = 8
                       ((8, 16, 32, 256, 2, 32, 4), stap.STAP_OK),          # D = 16
                       ((5, 16, 32, 256, 2, 32, 4), stap.STAP_OK),                 # D = 10
                       ((16, 16, 32, 256, 4, 32, 4), stap.STAP_OK),                # D = 64
                       ((11, 16, 32, 256, 3, 32, 4), stap.STAP_OK),                # D = 33
                       ((25, 16, 32, 256, 3, 32, 4), stap.STAP_OK),                # D = 75
                       ((43, 16, 32, 256, 3, 32, 4), stap.STAP_ERR_UNSUPPORTED)]:  # D = 129
        got, h, _ = _create(dims, mir)
        assert got == code, dims
        if h.value:
            stap.stap_plan_destroy(h)


def test_null_and_misaligned_pointers_and_missing_workspace_fail_before_cuda():
    L = stap.lib()
    h = ctypes.c_void_p()
    assert L.stap_plan_create(None, 1, None, None, ctypes.byref(h), None) == stap.STAP_ERR_INVALID_ARG
    code, h, ws = _create(GOOD)
    assert code == 0
    fake = ctypes.c_void_p(0x10000)                           # never dereferenced
    odd = ctypes.c_void_p(0x10008)
    step, run = stap.stap_plan_workspace_sizes(h)
    assert L.stap_plan_set_workspace(h, None, run) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_plan_set_workspace(h, odd, run) == stap.STAP_ERR_MISALIGNED
    assert L.stap_plan_set_workspace(h, fake, step - 1) == stap.STAP_ERR_NO_WORKSPACE
    # step calls: NULL -> invalid, misaligned -> misaligned, otherwise no workspace yet
    assert L.stap_doppler(h, None, fake) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_doppler(h, odd, fake) == stap.STAP_ERR_MISALIGNED
    assert L.stap_doppler(h, fake, fake) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_covariance(h, fake, fake) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_solve_weights(h, fake, fake) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_apply(h, fake, fake, fake) == stap.STAP_ERR_NO_WORKSPACE
    other = ctypes.c_void_p(0x20000)
    assert L.stap_train_neighbours(h, fake, fake) == stap.STAP_ERR_INVALID_ARG   # in place
    assert L.stap_train_neighbours(h, None, other) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_train_neighbours(h, odd, other) == stap.STAP_ERR_MISALIGNED
    assert L.stap_train_neighbours(h, fake, other) == stap.STAP_ERR_NO_WORKSPACE
    arr = (ctypes.c_void_p * 1)(fake)
    assert L.stap_run_cpi(h, arr, arr) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_get_status(h, None) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_plan_set_steering(h, 0, fake) == stap.STAP_ERR_NO_WORKSPACE
    assert L.stap_plan_set_steering(h, 1, fake) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_plan_destroy(None) == stap.STAP_ERR_INVALID_ARG
    stap.stap_plan_destroy(h)


def test_step_calls_need_a_single_cpi_plan():
    L = stap.lib()
    arr = (stap.stap_dims * 2)(stap.stap_dims(*GOOD), stap.stap_dims(4, 64, 64, 1024, 2, 64, 8))
    h = ctypes.c_void_p()
    assert L.stap_plan_create(arr, 2, None, None, ctypes.byref(h), None) == 0
    fake = ctypes.c_void_p(0x10000)
    assert L.stap_doppler(h, fake, fake) == stap.STAP_ERR_INVALID_ARG
    step, run = stap.stap_plan_workspace_sizes(h)
    assert run > step
    stap.stap_plan_destroy(h)


def test_status_strings():
    for code in range(9):
        s = stap.status_string(code)
        assert s and s != "unknown status"
    assert stap.status_string(99) == "unknown status"


def test_wait_limit_is_validated_without_cuda():
    L = stap.lib()
    code, h, _ = _create(GOOD)
    assert code == 0
    assert L.stap_plan_set_wait_limit(h, -1) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_plan_set_wait_limit(h, 0) == stap.STAP_OK
    assert L.stap_plan_set_wait_limit(h, stap.STAP_DEFAULT_WAIT_POLLS) == stap.STAP_OK
    assert L.stap_plan_set_wait_limit(None, 1) == stap.STAP_ERR_INVALID_ARG
    stap.stap_plan_destroy(h)


def test_check_report_is_unsupported_in_the_normal_build():
    assert not stap.stap_checked_build()
    with pytest.raises(stap.StapError) as e:
        stap.stap_check_report()
    assert e.value.code == stap.STAP_ERR_UNSUPPORTED


def test_checked_build_loads_and_exports_the_same_symbols():
    """The checked library (compiled with -DSTAP_CHECKED) loads without a GPU,
    says it is the checked build and exports every declared symbol."""
    import subprocess
    import sys
    code = ("from paper_2203_06233_gb300 import stap\n"
            "L = stap.lib()\n"
            "assert stap.lib_path().endswith('libstap_checked.so')\n"
            "assert stap.stap_checked_build()\n"
            "missing = [n for n in stap.EXPORTED if not hasattr(L, n)]\n"
            "assert not missing, missing\n"
            "print('checked ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, STAP_CHECKED="1"), timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout + r.stderr


def test_batch_schedule_values_without_cuda():
    L = stap.lib()
    arr = (stap.stap_dims * 2)(stap.stap_dims(*GOOD), stap.stap_dims(4, 64, 64, 1024, 2, 64, 8))
    h = ctypes.c_void_p()
    assert L.stap_plan_create(arr, 2, None, None, ctypes.byref(h), None) == 0
    assert stap.stap_plan_get_batch_schedule(h) == stap.STAP_BATCH_PERSISTENT
    assert L.stap_plan_set_batch_schedule(h, 2) == stap.STAP_ERR_INVALID_ARG
    stap.stap_plan_set_batch_schedule(h, stap.STAP_BATCH_STREAMS)
    assert stap.stap_plan_get_batch_schedule(h) == stap.STAP_BATCH_STREAMS
    stap.stap_plan_destroy(h)


def test_pivot_reciprocal_test_call_validates_before_any_cuda_call():
    L = stap.lib()
    assert L.stap_test_pivot_reciprocal(None, None, -1, None) == stap.STAP_ERR_INVALID_ARG
    assert L.stap_test_pivot_reciprocal(None, None, 4, None) == stap.STAP_ERR_INVALID_ARG
