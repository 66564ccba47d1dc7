"""FP64 CPU oracle for the STAP hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.

The arithmetic lives in ``stap_oracle.c`` (plain C99, IEEE double, OpenMP over
Doppler bins / systems).  This module only marshals numpy arrays into it.  The
definitions it follows, step by step (arXiv 2203.06233 Sec. 4.2, STAP kernel:
statement T is the `fft` over pulses, statement U the array multiply; the
remaining steps are the standard post-Doppler STAP reading):

1. ``doppler``     Hann-windowed direct DFT over pulses, zero-padded to K bins.
   ``doppler_staggered`` (an option beyond the paper): T sub-windows of
   P - T + 1 pulses, each transformed with its pulses' CPI phase; the result
   is a Doppler cube of C*T channels (``staggered_dims``) with one bin per
   snapshot, and ``default_steering_staggered`` its steering.
   ``reduce_channels`` (a front end beyond the paper): N element channels
   combined into C channels by a matrix W[C][N] (``subarray_weights``: C
   contiguous subarrays), with ``reduced_steering`` the matching steering.
2. ``snapshot``    D = C*T entries from T adjacent bins, channel fastest.
3. ``covariance``  R = (1/B) sum x x^H per (Doppler bin, range block).
   ``train_neighbours`` (an option beyond the paper): block b trained on the
   mean of the covariances of blocks b-1 and b+1, leaving out the cell under
   test and its block (guard cells).
4-7. ``weights``   diagonal load, Cholesky, forward/back solve, AMF scaling.
8. ``apply``       P = |w^H x|^2 per cell and steering vector.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, library routines and
brute force); none is "parity unpinned".
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class _Dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("n_chan", "n_pulses", "n_dop", "n_range", "tdof", "training_block", "n_steering")]


@dataclass(frozen=True)
class Dims:
    """Shape of one CPI: C channels, P pulses, K Doppler bins, R range cells,
    T adjacent-bin degrees of freedom, B-cell training blocks, S steering vectors."""
    n_chan: int
    n_pulses: int
    n_dop: int
    n_range: int
    tdof: int
    training_block: int
    n_steering: int

    @property
    def D(self) -> int:
        return self.n_chan * self.tdof

    @property
    def NB(self) -> int:
        return self.n_range // self.training_block

    def c(self, n_range=None) -> _Dims:
        return _Dims(self.n_chan, self.n_pulses, self.n_dop,
                     self.n_range if n_range is None else n_range,
                     self.tdof, self.training_block, self.n_steering)


def lib():
    global _lib
    if _lib is None:
        # STAP_ORACLE_LIB points the loader at another build of the same source
        # (the mutation tests load deliberately broken copies this way).
        path = os.environ.get("STAP_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32 = ctypes.c_int32
        D = ctypes.POINTER(_Dims)
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_hann.argtypes = [i32, P]
        L.oracle_hann.restype = None
        L.oracle_doppler_window.argtypes = [D, P, P, i32, i32, P]
        L.oracle_doppler.argtypes = [D, P, i32, i32, P]
        L.oracle_snapshot.argtypes = [D, P, i32, i32, i32, P]
        L.oracle_covariance.argtypes = [D, P, i32, P]
        L.oracle_cholesky.argtypes = [i32, P, P]
        L.oracle_cholesky_solve.argtypes = [i32, P, P, P]
        L.oracle_default_steering.argtypes = [D, P]
        L.oracle_weights.argtypes = [D, P, i32, P, ctypes.c_double, P, P]
        L.oracle_apply.argtypes = [D, P, i32, P, P]
        L.oracle_run.argtypes = [D, P, P, ctypes.c_double, i32, i32, P, P, P, P, P]
        L.oracle_train_neighbours.argtypes = [D, P, i32, i32, i32, P]
        L.oracle_run_neighbours.argtypes = [D, P, P, ctypes.c_double, i32, i32, P, P]
        L.oracle_train_window.argtypes = [D, P, i32, i32, i32, i32, i32, P]
        L.oracle_run_window.argtypes = [D, P, P, ctypes.c_double, i32, i32, i32, i32, P, P]
        L.oracle_doppler_staggered.argtypes = [D, P, i32, i32, P]
        L.oracle_default_steering_staggered.argtypes = [D, P]
        L.oracle_run_staggered.argtypes = [D, P, P, ctypes.c_double, i32, i32, P, P, P, P, P]
        L.oracle_reduce_channels.argtypes = [i32, i32, i32, i32, P, P, P]
        L.oracle_subarray_weights.argtypes = [i32, i32, P]
        L.oracle_reduced_steering.argtypes = [D, i32, P, P]
        for f in ("oracle_doppler_window", "oracle_doppler", "oracle_snapshot", "oracle_covariance",
                  "oracle_cholesky", "oracle_cholesky_solve", "oracle_default_steering",
                  "oracle_weights", "oracle_apply", "oracle_run", "oracle_train_neighbours",
                  "oracle_run_neighbours", "oracle_train_window", "oracle_run_window",
                  "oracle_doppler_staggered",
                  "oracle_default_steering_staggered", "oracle_run_staggered",
                  "oracle_reduce_channels", "oracle_subarray_weights", "oracle_reduced_steering"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
    return rc


def num_threads() -> int:
    return lib().oracle_num_threads()


def hann(P: int) -> np.ndarray:
    h = np.empty(P, np.float64)
    lib().oracle_hann(P, _ptr(h))
    return h


def _slab(d: Dims, cube, r0, nr):
    """The range cells [r0, r0+nr) of a [C][P][R] cube, promoted to complex128."""
    nr = d.n_range - r0 if nr is None else nr
    return nr, _c128(np.asarray(cube)[:, :, r0:r0 + nr])


def doppler(d: Dims, cube, r0=0, nr=None, window=None) -> np.ndarray:
    """dop[C][K][nr] of the range cells [r0, r0+nr) (step 1)."""
    nr, x = _slab(d, cube, r0, nr)
    out = np.empty((d.n_chan, d.n_dop, nr), np.complex128)
    if window is None:
        rc = lib().oracle_doppler(ctypes.byref(d.c(nr)), _ptr(x), 0, nr, _ptr(out))
    else:
        w = np.ascontiguousarray(window, np.float64)
        assert w.shape == (d.n_pulses,)
        rc = lib().oracle_doppler_window(ctypes.byref(d.c(nr)), _ptr(w), _ptr(x), 0, nr, _ptr(out))
    _check(rc, "doppler")
    return out


def snapshot(d: Dims, dop, k: int, r: int) -> np.ndarray:
    """x_{k,r} (D entries) from a Doppler window dop[C][K][nr] (step 2)."""
    dop = _c128(dop)
    nr = dop.shape[2]
    x = np.empty(d.D, np.complex128)
    _check(lib().oracle_snapshot(ctypes.byref(d.c()), _ptr(dop), nr, k, r, _ptr(x)), "snapshot")
    return x


def covariance(d: Dims, dop) -> np.ndarray:
    """cov[K][nr/B][D][D] from dop[C][K][nr] (step 3)."""
    dop = _c128(dop)
    nr = dop.shape[2]
    cov = np.empty((d.n_dop, nr // d.training_block, d.D, d.D), np.complex128)
    _check(lib().oracle_covariance(ctypes.byref(d.c()), _ptr(dop), nr, _ptr(cov)), "covariance")
    return cov


def cholesky(A) -> np.ndarray:
    """Lower L with A = L L^H (step 5); raises ValueError if A is not positive definite."""
    A = _c128(A)
    n = A.shape[0]
    L = np.empty_like(A)
    rc = _check(lib().oracle_cholesky(n, _ptr(A), _ptr(L)), "cholesky")
    if rc:
        raise ValueError(f"not positive definite at column {rc - 1}")
    return L


def cholesky_solve(L, b) -> np.ndarray:
    """u = (L L^H)^{-1} b (step 6)."""
    L = _c128(L)
    b = _c128(b)
    u = np.empty_like(b)
    _check(lib().oracle_cholesky_solve(L.shape[0], _ptr(L), _ptr(b), _ptr(u)), "cholesky_solve")
    return u


def default_steering(d: Dims) -> np.ndarray:
    """steer[S][D] (the default angle grid, window-matched temporal part)."""
    st = np.empty((d.n_steering, d.D), np.complex128)
    _check(lib().oracle_default_steering(ctypes.byref(d.c()), _ptr(st)), "default_steering")
    return st


def weights(d: Dims, cov, steer=None, load_factor=1e-3):
    """(wts[..][S][D], status[..], n_failed) for covariances cov[..][D][D] (steps 4-7)."""
    cov = _c128(cov)
    lead = cov.shape[:-2]
    nsys = int(np.prod(lead)) if lead else 1
    st = default_steering(d) if steer is None else _c128(steer)
    wts = np.empty(lead + (d.n_steering, d.D), np.complex128)
    status = np.empty(lead, np.int32)
    rc = _check(lib().oracle_weights(ctypes.byref(d.c()), _ptr(cov), nsys, _ptr(st),
                                     float(load_factor), _ptr(wts), _ptr(status)), "weights")
    return wts, status, rc


def apply(d: Dims, dop, wts) -> np.ndarray:
    """out[S][K][nr] = |w^H x|^2 (step 8)."""
    dop = _c128(dop)
    wts = _c128(wts)
    nr = dop.shape[2]
    out = np.empty((d.n_steering, d.n_dop, nr), np.float64)
    _check(lib().oracle_apply(ctypes.byref(d.c()), _ptr(dop), nr, _ptr(wts), _ptr(out)), "apply")
    return out


def train_neighbours(d: Dims, cov) -> np.ndarray:
    """Training matrices cov_t[K][NB][D][D] of neighbour-block training from the
    per-block covariances cov[K][NB][D][D] of a whole range (NB >= 2)."""
    cov = _c128(cov)
    K, nb = cov.shape[:2]
    out = np.empty_like(cov)
    _check(lib().oracle_train_neighbours(ctypes.byref(d.c()), _ptr(cov), nb, 0, nb, _ptr(out)),
           "train_neighbours")
    return out


def train_window(d: Dims, cov, guard: int, half: int) -> np.ndarray:
    """Training matrices cov_t[K][NG][D][D] of the sliding training window
    (``half`` groups on each side beyond ``guard`` guard groups) from the
    per-group covariances cov[K][NG][D][D] of a whole range."""
    cov = _c128(cov)
    K, nb = cov.shape[:2]
    out = np.empty_like(cov)
    _check(lib().oracle_train_window(ctypes.byref(d.c()), _ptr(cov), nb, 0, nb, int(guard), int(half),
                                     _ptr(out)), "train_window")
    return out


def reduce_channels(W, x) -> np.ndarray:
    """y[C][P][R] = sum_n conj(W[c][n]) x[n][P][R]: the reduced-DOF front end
    (N element channels of x combined into C channels by W[C][N])."""
    W, x = _c128(W), _c128(x)
    (C, N), (N2, P, R) = W.shape, x.shape
    assert N == N2
    y = np.empty((C, P, R), np.complex128)
    _check(lib().oracle_reduce_channels(N, C, P, R, _ptr(W), _ptr(x), _ptr(y)), "reduce_channels")
    return y


def subarray_weights(N: int, C: int) -> np.ndarray:
    """W[C][N] summing C contiguous subarrays of N / C elements."""
    W = np.empty((C, N), np.complex128)
    _check(lib().oracle_subarray_weights(N, C, _ptr(W)), "subarray_weights")
    return W


def reduced_steering(d: Dims, W) -> np.ndarray:
    """steer[S][D] of the channels reduced by W[C][N] (d.n_chan = C):
    v_s[t*C + c] = g_t sum_n conj(W[c][n]) exp(j 2 pi f_s n)."""
    W = _c128(W)
    assert W.shape[0] == d.n_chan
    st = np.empty((d.n_steering, d.D), np.complex128)
    _check(lib().oracle_reduced_steering(ctypes.byref(d.c()), W.shape[1], _ptr(W), _ptr(st)),
           "reduced_steering")
    return st


def staggered_dims(d: Dims) -> Dims:
    """The dims under which covariance, weights and apply see staggered
    snapshots: C*T channels, one bin (T = 1)."""
    return Dims(d.n_chan * d.tdof, d.n_pulses, d.n_dop, d.n_range, 1, d.training_block,
                d.n_steering)


def doppler_staggered(d: Dims, cube, r0=0, nr=None) -> np.ndarray:
    """Xs[T*C][K][nr]: sub-window t (pulses t .. t+P-T) of channel c in row t*C + c."""
    nr, x = _slab(d, cube, r0, nr)
    out = np.empty((d.tdof * d.n_chan, d.n_dop, nr), np.complex128)
    _check(lib().oracle_doppler_staggered(ctypes.byref(d.c(nr)), _ptr(x), 0, nr, _ptr(out)),
           "doppler_staggered")
    return out


def default_steering_staggered(d: Dims) -> np.ndarray:
    """steer[S][D] of staggered snapshots: v_s[t*C + c] = (sum h') a_c."""
    st = np.empty((d.n_steering, d.D), np.complex128)
    _check(lib().oracle_default_steering_staggered(ctypes.byref(d.c()), _ptr(st)),
           "default_steering_staggered")
    return st


def run(d: Dims, cube, r0=0, nr=None, steer=None, load_factor=1e-3, keep=False, training=0,
        staggered=False, guard=0, half=1):
    """Steps 1-8 on the range cells [r0, r0+nr) of a [C][P][R] cube.

    Returns a dict with ``out`` [S][K][nr] (float64), ``status`` [K][nr/B] and
    ``n_failed``; with ``keep`` also ``dop``, ``cov`` and ``wts``.  With
    ``training=1`` each block is trained on its neighbours (``train_neighbours``);
    the window is then computed from a slab one block wider on each side.  With
    ``training=2`` each group of B cells is trained on a sliding window
    (``train_window``: ``half`` groups on each side beyond ``guard`` guard
    groups), computed from a slab guard + half groups wider on each side.  With
    ``staggered`` the snapshots are PRI-staggered (``doppler_staggered``; ``dop``
    is then [T*C][K][nr]).
    """
    if training and staggered:
        raise ValueError("neighbour training with staggered snapshots is not defined here")
    if training == 2:
        if keep:
            raise ValueError("keep is not available with a training window")
        nr = d.n_range - r0 if nr is None else nr
        B = d.training_block
        if d.n_range // B < 2 * guard + 2 or half < 1 or guard < 0:
            raise ValueError("the training window needs half >= 1, guard >= 0, NB >= 2 guard + 2")
        ext = (guard + half) * B
        e0, e1 = max(0, r0 - ext), min(d.n_range, r0 + nr + ext)
        x = _c128(np.asarray(cube)[:, :, e0:e1])
        out = np.empty((d.n_steering, d.n_dop, nr), np.float64)
        status = np.empty((d.n_dop, nr // B), np.int32)
        st = None if steer is None else _c128(steer)
        rc = lib().oracle_run_window(ctypes.byref(d.c(e1 - e0)), _ptr(x),
                                     _ptr(st) if st is not None else ctypes.c_void_p(0),
                                     float(load_factor), r0 - e0, nr, int(guard), int(half),
                                     _ptr(out), _ptr(status))
        return {"out": out, "status": status, "n_failed": _check(rc, "run")}
    if training:
        if keep:
            raise ValueError("keep is not available with neighbour training")
        nr = d.n_range - r0 if nr is None else nr
        B = d.training_block
        e0, e1 = max(0, r0 - B), min(d.n_range, r0 + nr + B)
        x = _c128(np.asarray(cube)[:, :, e0:e1])
        out = np.empty((d.n_steering, d.n_dop, nr), np.float64)
        status = np.empty((d.n_dop, nr // B), np.int32)
        st = None if steer is None else _c128(steer)
        rc = lib().oracle_run_neighbours(ctypes.byref(d.c(e1 - e0)), _ptr(x),
                                         _ptr(st) if st is not None else ctypes.c_void_p(0),
                                         float(load_factor), r0 - e0, nr, _ptr(out), _ptr(status))
        return {"out": out, "status": status, "n_failed": _check(rc, "run")}
    nr, x = _slab(d, cube, r0, nr)
    NB = nr // d.training_block
    out = np.empty((d.n_steering, d.n_dop, nr), np.float64)
    status = np.empty((d.n_dop, NB), np.int32)
    res = {"out": out, "status": status}
    dop = cov = wts = None
    if keep:
        dop = res["dop"] = np.empty((d.D if staggered else d.n_chan, d.n_dop, nr), np.complex128)
        cov = res["cov"] = np.empty((d.n_dop, NB, d.D, d.D), np.complex128)
        wts = res["wts"] = np.empty((d.n_dop, NB, d.n_steering, d.D), np.complex128)
    st = None if steer is None else _c128(steer)
    nul = ctypes.c_void_p(0)
    fn = lib().oracle_run_staggered if staggered else lib().oracle_run
    rc = fn(ctypes.byref(d.c(nr)), _ptr(x), _ptr(st) if st is not None else nul,
                          float(load_factor), 0, nr,
                          _ptr(dop) if keep else nul, _ptr(cov) if keep else nul,
                          _ptr(wts) if keep else nul, _ptr(out), _ptr(status))
    res["n_failed"] = _check(rc, "run")
    return res
