"""Thin Python binding of libstap (the C ABI in ``include/stap.h``).

Argument marshalling only: every step of the STAP path runs in the CUDA
kernels of ``libstap.so``.  PyTorch provides device memory and streams.  The
functions carry the C names (``stap_plan_create``, ``stap_doppler``, ...) and
take torch tensors; :class:`Plan` wraps a plan together with its workspace.

If the compiled library is missing it is built with nvcc; if that fails an
error is raised -- there is no other implementation to fall back to.
"""
import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

STAP_OK = 0
STAP_ERR_INVALID_ARG = 1
STAP_ERR_SHAPE = 2
STAP_ERR_UNSUPPORTED = 3
STAP_ERR_CUDA = 4
STAP_ERR_NOT_POSDEF = 5
STAP_ERR_TIMEOUT = 6
STAP_ERR_NO_WORKSPACE = 7
STAP_ERR_MISALIGNED = 8

STAP_PREC_FP32 = 0
STAP_PREC_BF16X3 = 1
STAP_PREC_TF32X3 = 2
STAP_PREC_FP16_SCALED = 3
STAP_SOLVE_FP64 = 0
STAP_SOLVE_MIXED_IR = 1
STAP_TRAIN_OWN_BLOCK = 0
STAP_TRAIN_NEIGHBOURS = 1
STAP_TRAIN_WINDOW = 2
STAP_BATCH_PERSISTENT = 0
STAP_BATCH_STREAMS = 1
STAP_SNAP_ADJACENT_BINS = 0
STAP_SNAP_PRI_STAGGERED = 1

# every symbol include/stap.h declares
EXPORTED = (
    "stap_options_default", "stap_plan_create", "stap_plan_workspace_sizes",
    "stap_plan_set_workspace", "stap_plan_set_stream", "stap_plan_set_steering",
    "stap_plan_destroy", "stap_doppler", "stap_covariance", "stap_solve_weights", "stap_apply",
    "stap_run_cpi", "stap_get_status", "stap_status_string", "stap_abi_version",
    "stap_run_cpi_noalloc", "stap_plan_batch_bytes", "stap_plan_autotune", "stap_plan_get_tuning",
    "stap_plan_set_tuning", "stap_train_neighbours", "stap_plan_stream_bytes", "stap_run_stream",
    "stap_plan_set_front_end", "stap_reduce_channels", "stap_plan_set_wait_limit",
    "stap_train_window", "stap_checked_build", "stap_check_report", "stap_plan_set_batch_schedule",
    "stap_test_pivot_reciprocal",
    "stap_plan_get_batch_schedule",
)

STAP_TUNING_LEN = 9

# mbarrier polls before a tensor-core pipeline wait gives up (default)
STAP_DEFAULT_WAIT_POLLS = 4194304

# size of the library-owned scratch array used by stap_run_cpi_noalloc
STAP_NOALLOC_SCRATCH_BYTES = 16 << 20


class StapError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (status {code})")


class stap_dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("n_chan", "n_pulses", "n_dop", "n_range", "tdof", "training_block", "n_steering")]


class stap_options(ctypes.Structure):
    _fields_ = [("load_factor", ctypes.c_double), ("refine_steps", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("training", ctypes.c_int32), ("snapshots", ctypes.c_int32),
                ("train_guard", ctypes.c_int32), ("train_half", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def checked_requested() -> bool:
    """STAP_CHECKED=1 in the environment selects the checked build."""
    return os.environ.get("STAP_CHECKED", "") not in ("", "0")


def lib_path() -> str:
    return _build.LIB_CHECKED if checked_requested() else _build.LIB


_lib_tag = None


def lib_tag() -> str:
    """A short hash of the loaded library file: autotune cache entries are
    keyed by it, so a rebuilt library re-tunes instead of reusing choices
    timed on other kernels."""
    global _lib_tag
    if _lib_tag is None:
        import hashlib
        lib()
        with open(lib_path(), "rb") as f:
            _lib_tag = hashlib.sha256(f.read()).hexdigest()[:12]
    return _lib_tag


def lib():
    """Load libstap.so, or libstap_checked.so with STAP_CHECKED=1 (building it
    first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=checked_requested())
            L = ctypes.CDLL(path)
            vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
            L.stap_options_default.argtypes = [ctypes.POINTER(stap_options)]
            L.stap_options_default.restype = None
            L.stap_plan_create.argtypes = [ctypes.POINTER(stap_dims), i32, ctypes.POINTER(stap_options),
                                           vp, ctypes.POINTER(vp), ctypes.POINTER(sz)]
            L.stap_plan_workspace_sizes.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(sz)]
            L.stap_plan_set_workspace.argtypes = [vp, vp, sz]
            L.stap_plan_set_stream.argtypes = [vp, vp]
            L.stap_plan_set_wait_limit.argtypes = [vp, i32]
            L.stap_plan_set_steering.argtypes = [vp, i32, vp]
            L.stap_plan_destroy.argtypes = [vp]
            L.stap_doppler.argtypes = [vp, vp, vp]
            L.stap_covariance.argtypes = [vp, vp, vp]
            L.stap_solve_weights.argtypes = [vp, vp, vp]
            L.stap_train_neighbours.argtypes = [vp, vp, vp]
            L.stap_train_window.argtypes = [vp, vp, vp]
            L.stap_apply.argtypes = [vp, vp, vp, vp]
            L.stap_run_cpi.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
            L.stap_get_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
            L.stap_status_string.argtypes = [ctypes.c_int]
            L.stap_status_string.restype = ctypes.c_char_p
            L.stap_abi_version.argtypes = []
            L.stap_plan_batch_bytes.argtypes = [vp, ctypes.POINTER(sz)]
            L.stap_plan_stream_bytes.argtypes = [vp, ctypes.POINTER(sz)]
            L.stap_plan_set_front_end.argtypes = [vp, i32, vp, i32]
            L.stap_reduce_channels.argtypes = [vp, vp, vp]
            L.stap_run_stream.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(vp), ctypes.POINTER(vp)]
            L.stap_plan_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32]
            L.stap_plan_get_tuning.argtypes = [vp, i32, ctypes.POINTER(i32)]
            L.stap_plan_set_tuning.argtypes = [vp, i32, ctypes.POINTER(i32)]
            L.stap_checked_build.argtypes = []
            L.stap_test_pivot_reciprocal.argtypes = [vp, vp, ctypes.c_int64, vp]
            L.stap_plan_set_batch_schedule.argtypes = [vp, i32]
            L.stap_plan_get_batch_schedule.argtypes = [vp, ctypes.POINTER(i32)]
            L.stap_check_report.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i32),
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
            L.stap_run_cpi_noalloc.argtypes = [ctypes.POINTER(stap_dims), ctypes.POINTER(stap_options),
                                               vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
            for f in EXPORTED:
                if f not in ("stap_options_default", "stap_status_string"):
                    getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().stap_status_string(int(code)).decode()


def _check(code: int, what: str, ok=(STAP_OK,)):
    if code not in ok:
        raise StapError(code, what)
    return code


def _dims(d) -> stap_dims:
    if isinstance(d, stap_dims):
        return d
    if hasattr(d, "dims"):
        d = d.dims()
    return stap_dims(*[int(v) for v in d])


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# ------------------------------------------------------------- C entry points --

def stap_options_default() -> stap_options:
    o = stap_options()
    lib().stap_options_default(ctypes.byref(o))
    return o


def stap_plan_create(dims: Sequence, opts: Optional[stap_options] = None, stream=None):
    """(plan handle, run workspace bytes) for a list of CPI shapes."""
    arr = (stap_dims * len(dims))(*[_dims(d) for d in dims])
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check(lib().stap_plan_create(arr, len(dims), ctypes.byref(opts) if opts is not None else None,
                                  _stream_ptr(stream) if torch.cuda.is_available() else None,
                                  ctypes.byref(h), ctypes.byref(ws)), "stap_plan_create")
    return h, ws.value


def stap_plan_workspace_sizes(plan):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().stap_plan_workspace_sizes(plan, ctypes.byref(a), ctypes.byref(b)),
           "stap_plan_workspace_sizes")
    return a.value, b.value


def stap_plan_batch_bytes(plan) -> int:
    a = ctypes.c_size_t()
    _check(lib().stap_plan_batch_bytes(plan, ctypes.byref(a)), "stap_plan_batch_bytes")
    return a.value


def stap_plan_stream_bytes(plan) -> int:
    a = ctypes.c_size_t()
    _check(lib().stap_plan_stream_bytes(plan, ctypes.byref(a)), "stap_plan_stream_bytes")
    return a.value


def stap_plan_set_front_end(plan, W, chunk_elems: int = 0):
    """W: [C][N] complex (host); copied."""
    Wn = np.ascontiguousarray(np.asarray(W, dtype=np.complex128))
    _check(lib().stap_plan_set_front_end(plan, Wn.shape[1], Wn.ctypes.data_as(ctypes.c_void_p),
                                         int(chunk_elems)), "stap_plan_set_front_end")


def stap_reduce_channels(plan, elem_cube: torch.Tensor, cube: torch.Tensor):
    _check(lib().stap_reduce_channels(plan, ctypes.c_void_p(elem_cube.data_ptr()),
                                      ctypes.c_void_p(cube.data_ptr())), "stap_reduce_channels")


def stap_plan_set_workspace(plan, workspace: torch.Tensor):
    if not workspace.is_cuda or not workspace.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().stap_plan_set_workspace(plan, ctypes.c_void_p(workspace.data_ptr()), nbytes),
           "stap_plan_set_workspace")


def stap_plan_set_wait_limit(plan, max_polls: int):
    _check(lib().stap_plan_set_wait_limit(plan, int(max_polls)), "stap_plan_set_wait_limit")


def stap_plan_set_batch_schedule(plan, schedule: int):
    _check(lib().stap_plan_set_batch_schedule(plan, int(schedule)), "stap_plan_set_batch_schedule")


def stap_plan_get_batch_schedule(plan) -> int:
    v = ctypes.c_int32()
    _check(lib().stap_plan_get_batch_schedule(plan, ctypes.byref(v)), "stap_plan_get_batch_schedule")
    return v.value


def stap_plan_set_stream(plan, stream=None):
    _check(lib().stap_plan_set_stream(plan, _stream_ptr(stream)), "stap_plan_set_stream")


def stap_plan_set_steering(plan, cpi: int, steer):
    import numpy as np
    a = np.ascontiguousarray(steer, dtype=np.complex128)
    _check(lib().stap_plan_set_steering(plan, int(cpi), a.ctypes.data_as(ctypes.c_void_p)),
           "stap_plan_set_steering")


def stap_plan_destroy(plan):
    _check(lib().stap_plan_destroy(plan), "stap_plan_destroy")


def stap_doppler(plan, cube: torch.Tensor, dop: torch.Tensor):
    _check(lib().stap_doppler(plan, ctypes.c_void_p(cube.data_ptr()), ctypes.c_void_p(dop.data_ptr())),
           "stap_doppler")


def stap_covariance(plan, dop: torch.Tensor, cov: torch.Tensor):
    _check(lib().stap_covariance(plan, ctypes.c_void_p(dop.data_ptr()), ctypes.c_void_p(cov.data_ptr())),
           "stap_covariance")


def stap_train_neighbours(plan, cov: torch.Tensor, cov_train: torch.Tensor):
    _check(lib().stap_train_neighbours(plan, ctypes.c_void_p(cov.data_ptr()),
                                       ctypes.c_void_p(cov_train.data_ptr())), "stap_train_neighbours")


def stap_train_window(plan, cov: torch.Tensor, cov_train: torch.Tensor):
    _check(lib().stap_train_window(plan, ctypes.c_void_p(cov.data_ptr()),
                                   ctypes.c_void_p(cov_train.data_ptr())), "stap_train_window")


def stap_solve_weights(plan, cov: torch.Tensor, wts: torch.Tensor):
    _check(lib().stap_solve_weights(plan, ctypes.c_void_p(cov.data_ptr()),
                                    ctypes.c_void_p(wts.data_ptr())), "stap_solve_weights")


def stap_apply(plan, dop: torch.Tensor, wts: torch.Tensor, out: torch.Tensor):
    _check(lib().stap_apply(plan, ctypes.c_void_p(dop.data_ptr()), ctypes.c_void_p(wts.data_ptr()),
                            ctypes.c_void_p(out.data_ptr())), "stap_apply")


def stap_run_cpi(plan, cubes: Sequence[torch.Tensor], outs: Sequence[torch.Tensor]):
    n = len(cubes)
    ca = (ctypes.c_void_p * n)(*[t.data_ptr() for t in cubes])
    oa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
    _check(lib().stap_run_cpi(plan, ca, oa), "stap_run_cpi")


def stap_run_stream(plan, host_cubes: Sequence[torch.Tensor], host_outs: Sequence[torch.Tensor]):
    n = len(host_cubes)
    ca = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in host_cubes])
    oa = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in host_outs])
    _check(lib().stap_run_stream(plan, n, ca, oa), "stap_run_stream")


def stap_get_status(plan):
    """(status code, failed systems) -- waits for the plan's stream."""
    n = ctypes.c_int64()
    code = lib().stap_get_status(plan, ctypes.byref(n))
    _check(code, "stap_get_status", ok=(STAP_OK, STAP_ERR_NOT_POSDEF, STAP_ERR_TIMEOUT))
    return code, n.value


def stap_run_cpi_noalloc(dims, cube: torch.Tensor, out: torch.Tensor, opts=None, stream=None,
                         want_status: bool = False):
    """Whole chain for one CPI using the library's own fixed scratch array.

    For callers that must not allocate device memory: nothing is allocated
    here or in the library (``cube`` and ``out`` are the caller's).  With
    ``want_status`` the call waits for the stream and returns the number of
    covariances that were not positive definite; otherwise it returns None
    once the work is queued.
    """
    d = _dims(dims)
    n = ctypes.c_int64(0)
    code = lib().stap_run_cpi_noalloc(ctypes.byref(d), ctypes.byref(opts) if opts is not None else None,
                                      _stream_ptr(stream), ctypes.c_void_p(cube.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.byref(n) if want_status else None)
    _check(code, "stap_run_cpi_noalloc", ok=(STAP_OK, STAP_ERR_NOT_POSDEF) if want_status else (STAP_OK,))
    return n.value if want_status else None


def stap_plan_autotune(plan, cubes: Sequence[torch.Tensor], outs: Sequence[torch.Tensor], reps: int = 3):
    n = len(cubes)
    ca = (ctypes.c_void_p * n)(*[t.data_ptr() for t in cubes])
    oa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
    _check(lib().stap_plan_autotune(plan, ca, oa, int(reps)), "stap_plan_autotune")


def stap_plan_get_tuning(plan, cpi: int) -> List[int]:
    a = (ctypes.c_int32 * STAP_TUNING_LEN)()
    _check(lib().stap_plan_get_tuning(plan, int(cpi), a), "stap_plan_get_tuning")
    return list(a)


def stap_plan_set_tuning(plan, cpi: int, choices: Sequence[int]):
    a = (ctypes.c_int32 * STAP_TUNING_LEN)(*[int(v) for v in choices])
    _check(lib().stap_plan_set_tuning(plan, int(cpi), a), "stap_plan_set_tuning")


def default_tune_cache() -> str:
    return os.environ.get("STAP_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "stap_gb300", "tune.json")


def stap_abi_version() -> int:
    return lib().stap_abi_version()


def stap_test_pivot_reciprocal(x: torch.Tensor) -> torch.Tensor:
    """The factorisation's pivot reciprocal on a CUDA float64 tensor (test support)."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise StapError(STAP_ERR_INVALID_ARG, "stap_test_pivot_reciprocal: a CUDA float64 tensor")
    x = x.contiguous()
    out = torch.empty_like(x)
    _check(lib().stap_test_pivot_reciprocal(x.data_ptr(), out.data_ptr(), x.numel(),
                                            torch.cuda.current_stream(x.device).cuda_stream),
           "stap_test_pivot_reciprocal")
    return out


def stap_checked_build() -> bool:
    return lib().stap_checked_build() == 1


def stap_check_report():
    """(skipped accesses, site, index, extent) of the checked build, read and
    cleared; raises StapError (unsupported) on the normal build."""
    n, site, idx, ext = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().stap_check_report(ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx),
                                   ctypes.byref(ext)), "stap_check_report")
    return n.value, site.value, idx.value, ext.value


# --------------------------------------------------------------- convenience --

class Plan:
    """A libstap plan plus its torch-owned workspace, for tensors on one device.

    ``dims`` is one CPI shape (7 ints or an object with ``dims()``) or a list of
    them.  Calls are issued on torch's current stream.
    """

    def __init__(self, dims, load_factor: float = 1e-3, refine_steps: int = 1,
                 precision: int = STAP_PREC_FP32, device=None, steps_only: bool = False,
                 max_workspace_bytes: Optional[int] = None, solver: int = STAP_SOLVE_FP64,
                 training: int = STAP_TRAIN_OWN_BLOCK, snapshots: int = STAP_SNAP_ADJACENT_BINS,
                 front_end=None, front_end_chunk: int = 0, train_guard: int = 0, train_half: int = 1):
        dl = list(dims) if isinstance(dims, (list, tuple)) and dims and not isinstance(dims[0], int) \
            else [dims]
        self.dims = [_dims(d) for d in dl]
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        opts = stap_options(float(load_factor), int(refine_steps), int(precision), int(solver),
                            int(training), int(snapshots), int(train_guard), int(train_half))
        self.precision, self.refine_steps, self.solver = int(precision), int(refine_steps), int(solver)
        self.training, self.snapshots = int(training), int(snapshots)
        self.train_guard, self.train_half = int(train_guard), int(train_half)
        self.n_elem = 0
        with torch.cuda.device(self.device):
            self.handle, _ = stap_plan_create(self.dims, opts)
            if front_end is not None:   # N element channels -> C by W [C][N]
                stap_plan_set_front_end(self.handle, front_end, front_end_chunk)
                self.n_elem = int(np.asarray(front_end).shape[1])
            self.step_bytes, self.run_bytes = stap_plan_workspace_sizes(self.handle)
            self.batch_bytes = stap_plan_batch_bytes(self.handle)
            nbytes = self.step_bytes if steps_only else self.run_bytes
            if not steps_only and len(self.dims) > 1:
                # a batch: as much of the all-concurrent size as the cap allows
                cap = max_workspace_bytes if max_workspace_bytes is not None else 16 << 30
                nbytes = max(self.run_bytes, min(self.batch_bytes, cap))
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            stap_plan_set_workspace(self.handle, self.workspace)

    def close(self):
        if getattr(self, "handle", None) is not None:
            torch.cuda.synchronize(self.device)
            stap_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes of CPI i
    def shapes(self, i: int = 0):
        d = self.dims[i]
        C, P, K, R, T, B, S = (d.n_chan, d.n_pulses, d.n_dop, d.n_range, d.tdof,
                               d.training_block, d.n_steering)
        D, NB = C * T, R // B
        rows = D if self.snapshots == STAP_SNAP_PRI_STAGGERED else C   # Doppler rows
        sh = dict(cube=(C, P, R), dop=(rows, K, R), cov=(K, NB, D, D), wts=(K, NB, S, D),
                  out=(S, K, R))
        if self.n_elem:
            sh["elements"] = (self.n_elem, P, R)
        return sh

    def reduce_channels(self, elem_cube, cube=None):
        """The front end on the device: element cube [N][P][R] -> cube [C][P][R]."""
        sh = self.shapes()
        if not self.n_elem:
            raise ValueError("the plan has no front end")
        cube = torch.empty(sh["cube"], dtype=torch.complex64, device=self.device) if cube is None else cube
        _dev(elem_cube, torch.complex64, sh["elements"], "elem_cube")
        _dev(cube, torch.complex64, sh["cube"], "cube")
        self._sync_stream()
        stap_reduce_channels(self.handle, elem_cube, cube)
        return cube

    def _sync_stream(self):
        stap_plan_set_stream(self.handle, torch.cuda.current_stream(self.device))

    def doppler(self, cube, dop=None):
        sh = self.shapes()
        dop = torch.empty(sh["dop"], dtype=torch.complex64, device=self.device) if dop is None else dop
        _dev(cube, torch.complex64, sh["cube"], "cube")
        _dev(dop, torch.complex64, sh["dop"], "dop")
        self._sync_stream()
        stap_doppler(self.handle, cube, dop)
        return dop

    def covariance(self, dop, cov=None):
        sh = self.shapes()
        cov = torch.empty(sh["cov"], dtype=torch.complex128, device=self.device) if cov is None else cov
        _dev(dop, torch.complex64, sh["dop"], "dop")
        _dev(cov, torch.complex128, sh["cov"], "cov")
        self._sync_stream()
        stap_covariance(self.handle, dop, cov)
        return cov

    def train_neighbours(self, cov, cov_train=None):
        """Training matrices of STAP_TRAIN_NEIGHBOURS from per-block covariances."""
        sh = self.shapes()
        cov_train = torch.empty_like(cov) if cov_train is None else cov_train
        _dev(cov, torch.complex128, sh["cov"], "cov")
        _dev(cov_train, torch.complex128, sh["cov"], "cov_train")
        self._sync_stream()
        stap_train_neighbours(self.handle, cov, cov_train)
        return cov_train

    def train_window(self, cov, cov_train=None):
        """Training matrices of the sliding window (the plan's guard and half)."""
        sh = self.shapes()
        cov_train = torch.empty_like(cov) if cov_train is None else cov_train
        _dev(cov, torch.complex128, sh["cov"], "cov")
        _dev(cov_train, torch.complex128, sh["cov"], "cov_train")
        self._sync_stream()
        stap_train_window(self.handle, cov, cov_train)
        return cov_train

    def solve_weights(self, cov, wts=None):
        sh = self.shapes()
        wts = torch.empty(sh["wts"], dtype=torch.complex64, device=self.device) if wts is None else wts
        _dev(cov, torch.complex128, sh["cov"], "cov")
        _dev(wts, torch.complex64, sh["wts"], "wts")
        self._sync_stream()
        stap_solve_weights(self.handle, cov, wts)
        return wts

    def apply(self, dop, wts, out=None):
        sh = self.shapes()
        out = torch.empty(sh["out"], dtype=torch.float32, device=self.device) if out is None else out
        _dev(dop, torch.complex64, sh["dop"], "dop")
        _dev(wts, torch.complex64, sh["wts"], "wts")
        _dev(out, torch.float32, sh["out"], "out")
        self._sync_stream()
        stap_apply(self.handle, dop, wts, out)
        return out

    def run_cpi(self, cubes, outs=None) -> List[torch.Tensor]:
        single = isinstance(cubes, torch.Tensor)
        cubes = [cubes] if single else list(cubes)
        if len(cubes) != len(self.dims):
            raise ValueError(f"plan has {len(self.dims)} CPIs, got {len(cubes)} cubes")
        if outs is None:
            outs = [torch.empty(self.shapes(i)["out"], dtype=torch.float32, device=self.device)
                    for i in range(len(cubes))]
        elif isinstance(outs, torch.Tensor):
            outs = [outs]
        for i, (c, o) in enumerate(zip(cubes, outs)):
            sh = self.shapes(i)
            _dev(c, torch.complex64, sh["cube"], f"cubes[{i}]")
            _dev(o, torch.float32, sh["out"], f"outs[{i}]")
        self._sync_stream()
        stap_run_cpi(self.handle, cubes, outs)
        return outs[0] if single else outs

    def run_stream(self, host_cubes, host_outs=None) -> List[torch.Tensor]:
        """Stream host cubes through the whole chain (stap_run_stream): the
        copy-in of cube i+1 and the copy-out of result i-1 overlap the chain of
        cube i.  host_cubes: CPU complex64 tensors [C][P][R] (page-locked, e.g.
        ``pin_memory()``, for the copies to overlap); host_outs: CPU float32
        [S][K][R] (allocated page-locked when None).  Grows the workspace to
        stap_plan_stream_bytes on first use.  Returns once the work is queued on
        the current stream; synchronise it before reading host_outs or
        modifying host_cubes."""
        if len(self.dims) != 1:
            raise ValueError("run_stream needs a single-CPI plan")
        sh = self.shapes()
        host_cubes = list(host_cubes)
        if host_outs is None:
            host_outs = [torch.empty(sh["out"], dtype=torch.float32).pin_memory() for _ in host_cubes]
        host_outs = list(host_outs)
        if len(host_outs) != len(host_cubes):
            raise ValueError("host_outs and host_cubes differ in length")
        for i, (c, o) in enumerate(zip(host_cubes, host_outs)):
            _host(c, torch.complex64, sh["elements"] if self.n_elem else sh["cube"], f"host_cubes[{i}]")
            _host(o, torch.float32, sh["out"], f"host_outs[{i}]")
        need = stap_plan_stream_bytes(self.handle)
        if self.workspace.numel() < need:
            with torch.cuda.device(self.device):
                torch.cuda.synchronize(self.device)      # nothing still uses the old workspace
                self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
                stap_plan_set_workspace(self.handle, self.workspace)
        self._sync_stream()
        stap_run_stream(self.handle, host_cubes, host_outs)
        return host_outs

    def _tune_key(self, i: int) -> str:
        d = self.dims[i]
        key = "C%d P%d K%d T%d B%d S%d prec%d ref%d solve%d train%d" % (
            d.n_chan, d.n_pulses, d.n_dop, d.tdof, d.training_block, d.n_steering, self.precision,
            self.refine_steps, self.solver, self.training)
        if self.snapshots:
            key += " snap%d" % self.snapshots
        if self.training == STAP_TRAIN_WINDOW:
            key += " guard%d half%d" % (self.train_guard, self.train_half)
        key += " lib" + lib_tag()
        # a one-CPI plan also tunes its range slabs, which depend on R
        return key + (" R%d" % d.n_range if len(self.dims) == 1 else " batch")

    def autotune(self, cubes, outs=None, cache_path: Optional[str] = None, reps: int = 3,
                 force: bool = False) -> dict:
        """Pick launch choices per CPI shape: from the JSON cache at ``cache_path``
        (default ``$STAP_TUNE_CACHE`` or ``~/.cache/stap_gb300/tune.json``) when every
        shape is there, else by timing candidates on the device
        (``stap_plan_autotune``) and adding them to the cache.  Returns {key: choices}."""
        import json
        cubes = [cubes] if isinstance(cubes, torch.Tensor) else list(cubes)
        path = cache_path or default_tune_cache()
        cache = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        keys = [self._tune_key(i) for i in range(len(self.dims))]
        # a batch also keeps its schedule, keyed by all its CPI shapes
        import hashlib
        skey = None
        if len(self.dims) > 1:
            skey = "batch schedule prec%d %s" % (self.precision, hashlib.sha256(
                "|".join(self._tune_key(i) + " R%d" % self.dims[i].n_range
                         for i in range(len(self.dims))).encode()).hexdigest()[:16])
        if not force and all(len(cache.get(k, ())) == STAP_TUNING_LEN for k in keys) and \
                (skey is None or skey in cache):
            for i, k in enumerate(keys):
                stap_plan_set_tuning(self.handle, i, cache[k])
            if skey is not None:
                stap_plan_set_batch_schedule(self.handle, int(cache[skey]))
            return {k: cache[k] for k in keys}
        if outs is None:
            outs = [torch.empty(self.shapes(i)["out"], dtype=torch.float32, device=self.device)
                    for i in range(len(cubes))]
        elif isinstance(outs, torch.Tensor):
            outs = [outs]
        self._sync_stream()
        stap_plan_autotune(self.handle, cubes, outs, reps)
        result = {}
        for i, k in enumerate(keys):
            result[k] = cache[k] = stap_plan_get_tuning(self.handle, i)
        if skey is not None:
            cache[skey] = stap_plan_get_batch_schedule(self.handle)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".tmp.%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass
        return result

    def set_batch_schedule(self, schedule: int):
        """STAP_BATCH_PERSISTENT or STAP_BATCH_STREAMS for a batch plan."""
        stap_plan_set_batch_schedule(self.handle, schedule)

    def set_wait_limit(self, max_polls: int = STAP_DEFAULT_WAIT_POLLS):
        """Polls after which a tensor-core pipeline wait gives up (0: at once)."""
        stap_plan_set_wait_limit(self.handle, max_polls)

    def set_steering(self, steer, cpi: int = 0):
        self._sync_stream()
        stap_plan_set_steering(self.handle, cpi, steer)

    def status(self):
        return stap_get_status(self.handle)
