"""Pins for the FP64 CPU oracle: closed forms, invariants, library routines and
brute force, each chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a missing scale) fails one of them.

The paper (arXiv 2203.06233) prints no STAP numbers, so nothing here is a
value from it; the definitions pinned are the post-Doppler reading of its STAP
kernel (Sec. 4.2: `fft` over pulses, 2-D x 2-D array multiply).
"""
import dataclasses
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2203_06233_gb300 import synth

RNG = np.random.default_rng(12345)


def crandn(*shape):
    return (RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)) / np.sqrt(2.0)


def dims(C=3, P=16, K=16, R=64, T=3, B=16, S=4):
    return oracle.Dims(C, P, K, R, T, B, S)


# ---------------------------------------------------------------- window -----

@pytest.mark.parametrize("P", [1, 2, 5, 32, 128])
def test_hann_is_numpy_symmetric_hann(P):
    h = oracle.hann(P)
    np.testing.assert_allclose(h, np.hanning(P), rtol=0, atol=1e-15)
    np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-15)
    if P > 1:
        assert h[0] == 0.0 and abs(h[-1]) < 1e-16


# ---------------------------------------------------------------- doppler ----

def _geom(w, P):
    """sum_{p<P} w^p in closed form."""
    if abs(w - 1.0) < 1e-14:
        return complex(P)
    return (1.0 - w ** P) / (1.0 - w)


@pytest.mark.parametrize("P,K,k0", [(32, 32, 5), (20, 64, 61), (33, 64, 0)])
def test_doppler_tone_on_bin_closed_form(P, K, k0):
    """x[p] = exp(j 2 pi k0 p / K): X[k] = sum_p h[p] exp(-j 2 pi (k-k0) p / K),
    with the Hann sum expanded into three geometric series."""
    d = dims(C=2, P=P, K=K, R=4, T=1, B=4, S=1)
    p = np.arange(P)
    tone = np.exp(2j * np.pi * k0 * p / K)
    cube = np.broadcast_to(tone[None, :, None], (2, P, 4)).astype(np.complex128)
    X = oracle.doppler(d, cube)
    th = 2.0 * np.pi / (P - 1)
    for k in range(K):
        z = np.exp(-2j * np.pi * (k - k0) / K)
        ref = 0.5 * _geom(z, P) - 0.25 * _geom(z * np.exp(1j * th), P) \
            - 0.25 * _geom(z * np.exp(-1j * th), P)
        np.testing.assert_allclose(X[:, k, :], ref, rtol=0, atol=1e-12 * P)


def test_doppler_matches_numpy_fft_with_zero_padding():
    d = dims(C=3, P=24, K=64, R=40, T=1, B=8, S=1)
    cube = crandn(3, 24, 40)
    ref = np.fft.fft(np.hanning(24)[None, :, None] * cube, n=64, axis=1)
    X = oracle.doppler(d, cube)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-13


def test_doppler_linearity_and_parseval_rect_window():
    d = dims(C=2, P=16, K=16, R=8, T=1, B=8, S=1)
    x, y = crandn(2, 16, 8), crandn(2, 16, 8)
    a, b = 0.3 - 1.2j, -2.0 + 0.5j
    lhs = oracle.doppler(d, a * x + b * y)
    rhs = a * oracle.doppler(d, x) + b * oracle.doppler(d, y)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13
    X = oracle.doppler(d, x, window=np.ones(16))
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2, axis=1), 16 * np.sum(np.abs(x) ** 2, axis=1),
                               rtol=1e-12)


def test_doppler_range_window_is_a_slice():
    d = dims(C=2, P=8, K=16, R=32, T=1, B=8, S=1)
    x = crandn(2, 8, 32)
    full = oracle.doppler(d, x)
    part = oracle.doppler(d, x, r0=8, nr=16)
    np.testing.assert_array_equal(part, full[:, :, 8:24])


# ---------------------------------------------------------------- snapshot ---

@pytest.mark.parametrize("T", [1, 2, 3, 4])
def test_snapshot_index_mapping(T):
    """dop values encode their own (c, k, r): the snapshot must read channel c
    of bin (k + t - floor(T/2)) mod K at entry t*C + c."""
    C, K, R = 3, 8, 5
    d = dims(C=C, P=8, K=K, R=R, T=T, B=5, S=1)
    c, k, r = np.meshgrid(np.arange(C), np.arange(K), np.arange(R), indexing="ij")
    dop = (c + 10 * k + 1000 * r) + 1j * (r - c)
    for kk in (0, 1, K - 1):
        for rr in (0, R - 1):
            x = oracle.snapshot(d, dop, kk, rr)
            for t in range(T):
                for cc in range(C):
                    kb = (kk + t - T // 2) % K
                    assert x[t * C + cc] == (cc + 10 * kb + 1000 * rr) + 1j * (rr - cc)


# ---------------------------------------------------------------- covariance -

def _gather(dop, T):
    """x[k, r, t*C + c] = dop[c, (k + t - T//2) % K, r], by numpy indexing."""
    C, K, R = dop.shape
    x = np.empty((K, R, T * C), np.complex128)
    for t in range(T):
        kk = (np.arange(K) + t - T // 2) % K
        x[:, :, t * C:(t + 1) * C] = dop[:, kk, :].transpose(1, 2, 0)
    return x


def test_covariance_equals_blocked_outer_products():
    d = dims(C=3, P=8, K=8, R=48, T=3, B=16, S=1)
    dop = crandn(3, 8, 48)
    cov = oracle.covariance(d, dop)
    x = _gather(dop, 3).reshape(8, 3, 16, 9)                    # [K][NB][B][D]
    ref = np.einsum("kbri,kbrj->kbij", x, x.conj()) / 16
    assert cov.shape == (8, 3, 9, 9)
    assert np.max(np.abs(cov - ref)) < 1e-13 * np.max(np.abs(ref))


def test_covariance_hermitian_psd_trace_rank():
    d = dims(C=2, P=4, K=4, R=12, T=3, B=4, S=1)                 # B=4 < D=6
    dop = crandn(2, 4, 12) * 10.0
    cov = oracle.covariance(d, dop)
    x = _gather(dop, 3).reshape(4, 3, 4, 6)
    for k in range(4):
        for b in range(3):
            Rm = cov[k, b]
            np.testing.assert_array_equal(Rm, Rm.conj().T)
            ev = np.linalg.eigvalsh(Rm)
            tr = np.trace(Rm).real
            assert ev.min() > -1e-12 * tr
            assert np.sum(ev > 1e-10 * tr) <= 4                 # rank <= B
            np.testing.assert_allclose(tr, np.mean(np.sum(np.abs(x[k, b]) ** 2, axis=1)),
                                       rtol=1e-13)


def _true_covariance(d, cnr_db, k):
    """Covariance of the snapshot at bin k under the synthetic data model:
    unit white noise through the window plus the 64-patch clutter ridge."""
    C, P, K, T = d.n_chan, d.n_pulses, d.n_dop, d.tdof
    h = np.hanning(P)
    p = np.arange(P)
    m = np.arange(T) - T // 2
    Rn = np.zeros((T * C, T * C), np.complex128)
    for t1 in range(T):
        for t2 in range(T):
            val = np.sum(h * h * np.exp(-2j * np.pi * p * (m[t1] - m[t2]) / K))
            for c in range(C):
                Rn[t1 * C + c, t2 * C + c] = val
    f = synth.patch_frequencies()
    Rc = np.zeros_like(Rn)
    for fi in f:
        Hb = np.array([np.sum(h * np.exp(2j * np.pi * p * (fi - (k + mt) / K))) for mt in m])
        z = (Hb[:, None] * np.exp(2j * np.pi * fi * np.arange(C))[None, :]).reshape(-1)
        Rc += (10 ** (cnr_db / 10) / synth.N_PATCH) * np.outer(z, z.conj())
    return Rn + Rc


def test_covariance_converges_to_data_model_covariance():
    """With one long training block the estimate approaches the analytic
    covariance of noise + clutter ridge; a sign slip in the DFT, a wrong bin
    offset or a missing 1/B fails this by orders of magnitude."""
    spec = synth.CPISpec(2, 16, 16, 8192, 3, 8192, 1, cnr_db=10.0, seed=77)
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    dop = oracle.doppler(d, cube)
    cov = oracle.covariance(d, dop)
    for k in (0, 3, 8, 13):
        Rt = _true_covariance(d, 10.0, k)
        err = np.linalg.norm(cov[k, 0] - Rt) / np.linalg.norm(Rt)
        assert err < 5.0 / np.sqrt(8192), (k, err)


# ---------------------------------------------------------------- cholesky ---

def _hpd(n, cond=1e3):
    Q, _ = np.linalg.qr(crandn(n, n))
    ev = np.logspace(0, np.log10(cond), n)
    return (Q * ev) @ Q.conj().T


@pytest.mark.parametrize("n", [1, 2, 7, 12, 33])
def test_cholesky_reconstructs_and_matches_numpy(n):
    A = _hpd(n)
    A = 0.5 * (A + A.conj().T)
    L = oracle.cholesky(A)
    assert np.all(np.triu(L, 1) == 0)
    assert np.all(np.diag(L).real > 0) and np.all(np.diag(L).imag == 0)
    assert np.linalg.norm(L @ L.conj().T - A) / np.linalg.norm(A) < 1e-12
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-11 * np.abs(L).max())


def test_cholesky_rejects_indefinite():
    A = np.diag([2.0, -1.0, 3.0]).astype(np.complex128)
    with pytest.raises(ValueError, match="column 1"):
        oracle.cholesky(A)


class _Q:
    """Exact complex rational."""

    def __init__(self, re, im=0):
        self.re, self.im = Fraction(re), Fraction(im)

    def __add__(self, o):
        return _Q(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return _Q(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        return _Q(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    def __truediv__(self, o):
        den = o.re * o.re + o.im * o.im
        return _Q((self.re * o.re + self.im * o.im) / den, (self.im * o.re - self.re * o.im) / den)

    def is_zero(self):
        return self.re == 0 and self.im == 0


def _exact_solve(A, b):
    """Gauss-Jordan elimination in exact rational arithmetic."""
    n = len(b)
    M = [[_Q(int(A[i, j].real), int(A[i, j].imag)) for j in range(n)] +
         [_Q(int(b[i].real), int(b[i].imag))] for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if not M[r][col].is_zero())
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [v / pv for v in M[col]]
        for r in range(n):
            if r != col and not M[r][col].is_zero():
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return np.array([float(M[i][n].re) + 1j * float(M[i][n].im) for i in range(n)])


@pytest.mark.parametrize("n", [2, 4, 6])
def test_cholesky_solve_matches_exact_rational_solution(n):
    rng = np.random.default_rng(n)
    M = rng.integers(-3, 4, (n, n)) + 1j * rng.integers(-3, 4, (n, n))
    A = M @ M.conj().T + n * np.eye(n)                           # Gaussian-integer HPD
    b = rng.integers(-5, 6, n) + 1j * rng.integers(-5, 6, n)
    u = oracle.cholesky_solve(oracle.cholesky(A), b)
    ref = _exact_solve(A, b)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-13
    np.testing.assert_allclose(u, np.linalg.solve(A, b), rtol=1e-12)


# ---------------------------------------------------------------- steering ---

@pytest.mark.parametrize("C,P,K,T,S,s0,k0", [(4, 32, 32, 3, 4, 2, 24), (3, 20, 64, 4, 5, 0, 1),
                                              (2, 16, 16, 2, 3, 1, 15)])
def test_default_steering_is_noise_free_target_snapshot(C, P, K, T, S, s0, k0):
    """A unit target at a bin centre on the steering grid has snapshot v_{s0}."""
    spec = synth.CPISpec(C, P, K, 8, T, 8, S, cnr_db=None, noise=False,
                         targets=(synth.Target(5, k0, s0, 0.0, 0.0),))
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec).astype(np.complex128)
    # regenerate the target in float64 to avoid the complex64 rounding of the cube
    th = np.deg2rad(synth.steering_angle_deg(s0, S))
    cube[:, :, 5] = np.exp(2j * np.pi * 0.5 * np.sin(th) * np.arange(C))[:, None] * \
        np.exp(2j * np.pi * k0 / K * np.arange(P))[None, :]
    dop = oracle.doppler(d, cube)
    x = oracle.snapshot(d, dop, k0, 5)
    v = oracle.default_steering(d)[s0]
    np.testing.assert_allclose(x, v, rtol=0, atol=1e-12 * np.abs(v).max())


def test_default_steering_angles_and_temporal_part():
    d = dims(C=5, P=12, K=24, T=3, S=6)
    st = oracle.default_steering(d)
    h = np.hanning(12)
    for s in range(6):
        th = np.deg2rad(-90 + 180 * (s + 0.5) / 6)
        a = np.exp(2j * np.pi * 0.5 * np.sin(th) * np.arange(5))
        g = np.array([np.sum(h * np.exp(-2j * np.pi * m * np.arange(12) / 24)) for m in (-1, 0, 1)])
        np.testing.assert_allclose(st[s], np.kron(g, a), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- weights ----

def test_weights_white_noise_closed_form():
    """R = sigma^2 I: w_s = v_s / (sigma sqrt(1 + lf) ||v_s||)."""
    d = dims(C=3, P=16, K=16, T=2, S=5)
    sig2, lf = 2.5, 1e-3
    cov = np.broadcast_to(sig2 * np.eye(6), (4, 6, 6)).astype(np.complex128)
    w, status, nf = oracle.weights(d, cov, load_factor=lf)
    assert nf == 0 and np.all(status == 0)
    v = oracle.default_steering(d)
    ref = v / (np.sqrt(sig2 * (1 + lf)) * np.linalg.norm(v, axis=1, keepdims=True))
    for i in range(4):
        np.testing.assert_allclose(w[i], ref, rtol=1e-13)


def test_weights_unit_noise_gain_and_optimal_sinr():
    """w = R^{-1} v / sqrt(v^H R^{-1} v): w^H R w = 1 and |w^H v|^2 = v^H R^{-1} v
    (the optimal output SINR for a unit target), here with no loading."""
    d = dims(C=2, P=8, K=8, T=3, S=3)
    R = _hpd(6, cond=1e4)
    R = 0.5 * (R + R.conj().T)
    steer = crandn(3, 6)
    w, _, _ = oracle.weights(d, R[None], steer=steer, load_factor=0.0)
    for s in range(3):
        ws = w[0, s]
        np.testing.assert_allclose((ws.conj() @ R @ ws).real, 1.0, rtol=1e-10)
        sinr = np.real(steer[s].conj() @ np.linalg.solve(R, steer[s]))
        np.testing.assert_allclose(np.abs(ws.conj() @ steer[s]) ** 2, sinr, rtol=1e-10)


def test_weights_loading_uses_trace_over_D():
    d = dims(C=2, P=8, K=8, T=1, S=2)
    R = _hpd(2)
    R = 0.5 * (R + R.conj().T)
    steer = crandn(2, 2)
    lf = 0.37
    w, _, _ = oracle.weights(d, R[None], steer=steer, load_factor=lf)
    Rl = R + lf * np.trace(R).real / 2 * np.eye(2)
    for s in range(2):
        u = np.linalg.solve(Rl, steer[s])
        np.testing.assert_allclose(w[0, s], u / np.sqrt(np.real(steer[s].conj() @ u)), rtol=1e-12)


def test_weights_flag_indefinite_system():
    d = dims(C=1, P=8, K=8, T=2, S=2)
    good = np.eye(2, dtype=np.complex128)
    bad = np.diag([1.0, -5.0]).astype(np.complex128)
    w, status, nf = oracle.weights(d, np.stack([good, bad, good]), load_factor=0.0)
    assert nf == 1 and list(status) == [0, 2, 0]
    assert np.all(w[1] == 0) and np.all(np.isfinite(w))


# ---------------------------------------------------------------- apply ------

def test_apply_matches_einsum_and_unit_vector_weights():
    d = dims(C=2, P=8, K=8, R=32, T=2, B=8, S=3)
    dop = crandn(2, 8, 32)
    wts = crandn(8, 4, 3, 4)
    out = oracle.apply(d, dop, wts)
    x = _gather(dop, 2)                                         # [K][R][D]
    wb = np.repeat(wts, 8, axis=1)                              # [K][R][S][D]
    ref = np.abs(np.einsum("krsd,krd->skr", wb.conj(), x)) ** 2
    np.testing.assert_allclose(out, ref, rtol=1e-12)
    e = np.zeros((8, 4, 3, 4), np.complex128)
    e[..., 0, 1] = 1.0                                          # steering 0 picks entry 1
    out = oracle.apply(d, dop, e)
    np.testing.assert_allclose(out[0], np.abs(x[:, :, 1]) ** 2, rtol=1e-15)
    assert np.all(out[1:] == 0)


# ---------------------------------------------------------------- whole path -

def test_run_is_composition_of_steps_and_windows_are_slices():
    spec = synth.CPISpec(3, 16, 32, 128, 3, 32, 4, cnr_db=30.0,
                         targets=(synth.Target(40, 7, 1, 10.0),), seed=9)
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    res = oracle.run(d, cube, keep=True)
    dop = oracle.doppler(d, cube)
    cov = oracle.covariance(d, dop)
    w, _, _ = oracle.weights(d, cov)
    out = oracle.apply(d, dop, w)
    np.testing.assert_array_equal(res["dop"], dop)
    np.testing.assert_array_equal(res["cov"], cov)
    np.testing.assert_array_equal(res["wts"], w)
    np.testing.assert_array_equal(res["out"], out)
    part = oracle.run(d, cube, r0=64, nr=32)
    np.testing.assert_array_equal(part["out"], res["out"][:, :, 64:96])


def test_small_workload_recovers_injected_target():
    """The small workload's 10 dB target at (range 128, bin 24, steering 2) is the
    strongest cell of its Doppler/steering row and > 10 dB above the median."""
    spec = synth.small_cpi()
    d = oracle.Dims(*spec.dims())
    res = oracle.run(d, synth.make_cube(spec))
    P = res["out"]
    assert res["n_failed"] == 0
    assert int(np.argmax(P[2, 24])) == 128
    assert 10 * np.log10(P[2, 24, 128] / np.median(P)) > 10.0


def test_noise_only_output_mean_near_one():
    """AMF output on noise alone has mean close to 1 (a little below, since the
    cell under test is part of its own training block)."""
    spec = synth.CPISpec(4, 32, 32, 4096, 3, 256, 4, cnr_db=None, seed=21)
    d = oracle.Dims(*spec.dims())
    P = oracle.run(d, synth.make_cube(spec))["out"]
    assert 0.85 < P.mean() < 1.05, P.mean()


# ------------------------------------------- training with guard cells ------

def test_neighbour_training_is_the_covariance_of_the_adjacent_blocks_cells():
    """Block b's training matrix is the sample covariance of the cells of blocks
    b-1 and b+1 (only the one that exists at either end), computed here from the
    gathered snapshots of exactly those cells."""
    d = dims(C=2, P=8, K=8, R=80, T=3, B=16, S=1)                # NB = 5
    dop = crandn(2, 8, 80)
    got = oracle.train_neighbours(d, oracle.covariance(d, dop))
    x = _gather(dop, 3)                                          # [K][R][D]
    for b in range(5):
        cells = [r for nb in (b - 1, b + 1) if 0 <= nb < 5 for r in range(16 * nb, 16 * nb + 16)]
        xs = x[:, cells]
        ref = np.einsum("kri,krj->kij", xs, xs.conj()) / len(cells)
        assert np.max(np.abs(got[:, b] - ref)) < 1e-13 * np.max(np.abs(ref)), b


def test_neighbour_training_run_composes_and_windows_are_slices():
    spec = synth.CPISpec(3, 16, 32, 128, 3, 32, 4, cnr_db=30.0,
                         targets=(synth.Target(40, 7, 1, 10.0),), seed=9)
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    full = oracle.run(d, cube, training=1)
    dop = oracle.doppler(d, cube)
    w, _, _ = oracle.weights(d, oracle.train_neighbours(d, oracle.covariance(d, dop)))
    np.testing.assert_array_equal(full["out"], oracle.apply(d, dop, w))
    for r0, nr in ((0, 32), (32, 64), (96, 32)):               # ends and middle
        part = oracle.run(d, cube, r0=r0, nr=nr, training=1)
        np.testing.assert_array_equal(part["out"], full["out"][:, :, r0:r0 + nr])


def test_neighbour_training_keeps_the_target_out_of_its_own_training():
    """The small workload's target trains its own block's weights, which then
    partly null it; trained on the neighbouring blocks its output stands more
    than four times higher above the median, and is still its row's maximum."""
    spec = synth.small_cpi()
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    own = oracle.run(d, cube)["out"]
    nbr = oracle.run(d, cube, training=1)["out"]
    assert int(np.argmax(nbr[2, 24])) == 128
    ratio_own = own[2, 24, 128] / np.median(own)
    ratio_nbr = nbr[2, 24, 128] / np.median(nbr)
    assert ratio_nbr > 4 * ratio_own, (ratio_own, ratio_nbr)


def test_neighbour_training_noise_only_output_mean_above_one():
    """With the cell under test outside its training data the AMF output on
    noise alone averages a little above 1 (about N / (N - D) for N training
    cells), where own-block training stays at or below 1."""
    spec = synth.CPISpec(4, 32, 32, 4096, 3, 256, 4, cnr_db=None, seed=21)
    d = oracle.Dims(*spec.dims())
    P = oracle.run(d, synth.make_cube(spec), training=1)["out"]
    assert 1.0 < P.mean() < 1.1, P.mean()


# --------------------------------------------- sliding training window ----
# Group j (B cells; B = 1: one cell) trains on the `half` groups on each side
# beyond `guard` guard groups, dropping groups outside the range.

@pytest.mark.parametrize("B,guard,half", [(1, 2, 6), (4, 1, 3), (16, 0, 1), (8, 2, 1)])
def test_training_window_is_the_covariance_of_exactly_its_training_cells(B, guard, half):
    """Group j's training matrix is the sample covariance of the cells of
    groups j-guard-half .. j-guard-1 and j+guard+1 .. j+guard+half that exist,
    computed here from the gathered snapshots of exactly those cells."""
    R = 96
    NG = R // B
    d = dims(C=2, P=8, K=8, R=R, T=3, B=B, S=1)
    dop = crandn(2, 8, R)
    got = oracle.train_window(d, oracle.covariance(d, dop), guard, half)
    x = _gather(dop, 3)                                          # [K][R][D]
    for j in range(NG):
        groups = [i for i in list(range(j - guard - half, j - guard)) +
                  list(range(j + guard + 1, j + guard + half + 1)) if 0 <= i < NG]
        assert groups and j not in groups
        cells = [r for i in groups for r in range(B * i, B * i + B)]
        xs = x[:, cells]
        ref = np.einsum("kri,krj->kij", xs, xs.conj()) / len(cells)
        assert np.max(np.abs(got[:, j] - ref)) < 1e-13 * np.max(np.abs(ref)), j


def test_training_window_reduces_to_neighbour_blocks_and_rejects_short_ranges():
    d = dims(C=2, P=8, K=8, R=80, T=3, B=16, S=1)                # NB = 5
    cov = oracle.covariance(d, crandn(2, 8, 80))
    np.testing.assert_array_equal(oracle.train_window(d, cov, 0, 1), oracle.train_neighbours(d, cov))
    with pytest.raises(RuntimeError):
        oracle.train_window(d, cov, 2, 1)                        # NB = 5 < 2 guard + 2
    with pytest.raises(RuntimeError):
        oracle.train_window(d, cov, 0, 0)


def test_training_window_run_composes_and_windows_are_slices():
    spec = synth.CPISpec(3, 16, 32, 128, 3, 4, 4, cnr_db=30.0,
                         targets=(synth.Target(40, 7, 1, 10.0),), seed=9)
    d = oracle.Dims(*spec.dims())
    cube = synth.make_cube(spec)
    full = oracle.run(d, cube, training=2, guard=1, half=4)
    dop = oracle.doppler(d, cube)
    w, _, _ = oracle.weights(d, oracle.train_window(d, oracle.covariance(d, dop), 1, 4))
    np.testing.assert_array_equal(full["out"], oracle.apply(d, dop, w))
    for r0, nr in ((0, 8), (40, 24), (120, 8), (0, 128)):       # ends, middle, whole
        part = oracle.run(d, cube, r0=r0, nr=nr, training=2, guard=1, half=4)
        np.testing.assert_array_equal(part["out"], full["out"][:, :, r0:r0 + nr])


def test_per_cell_training_window_keeps_the_target_out_of_its_own_training():
    """Per-cell windows (B = 1) with a guard of 2 cells on each side and 16
    training cells on each side: the small workload's target no longer trains
    its own weights, so its output stands far higher above the median than
    with own-block training (and above the neighbour-block form's), and is its
    row's maximum."""
    spec = synth.small_cpi()
    cube = synth.make_cube(spec)
    own = oracle.run(oracle.Dims(*spec.dims()), cube)["out"]
    nbr = oracle.run(oracle.Dims(*spec.dims()), cube, training=1)["out"]
    cell = dataclasses.replace(spec, training_block=1)
    win = oracle.run(oracle.Dims(*cell.dims()), cube, training=2, guard=2, half=16)["out"]
    assert int(np.argmax(win[2, 24])) == 128
    ratio_own = own[2, 24, 128] / np.median(own)
    ratio_nbr = nbr[2, 24, 128] / np.median(nbr)
    ratio_win = win[2, 24, 128] / np.median(win)
    print(f"target over median: own block {ratio_own:.1f}, neighbour blocks {ratio_nbr:.1f}, "
          f"per-cell window {ratio_win:.1f}")
    assert ratio_win > 4 * ratio_own and ratio_win > ratio_nbr, (ratio_own, ratio_nbr, ratio_win)


# ------------------------------------------------- PRI-staggered snapshots ----
# T sub-windows of P' = P - T + 1 pulses (sub-window t starts at pulse t), each
# Hann(P')-windowed and transformed with its pulses' CPI phase; the snapshot of
# bin k takes bin k of every sub-window.

def _shifted_windows(P, T):
    """win[t][p] = h'[p - t] on t <= p < t + P', else 0 (h' = numpy Hann of P')."""
    Ps = P - T + 1
    win = np.zeros((T, P))
    for t in range(T):
        win[t, t:t + Ps] = np.hanning(Ps)
    return win


@pytest.mark.parametrize("C,P,K,T", [(3, 16, 16, 3), (2, 20, 64, 4), (4, 9, 16, 2), (1, 5, 8, 5)])
def test_staggered_doppler_is_numpy_fft_of_shifted_windows(C, P, K, T):
    d = dims(C=C, P=P, K=K, R=24, T=T, B=8)
    cube = crandn(C, P, 24)
    xs = oracle.doppler_staggered(d, cube)
    win = _shifted_windows(P, T)
    for t in range(T):
        ref = np.fft.fft(win[t][None, :, None] * cube, n=K, axis=1)
        np.testing.assert_allclose(xs[t * C:(t + 1) * C], ref, rtol=0,
                                   atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("C,P,K,T,S,s0,k0", [(4, 32, 32, 3, 4, 2, 24), (3, 20, 64, 4, 5, 0, 1),
                                              (2, 16, 16, 2, 3, 1, 15)])
def test_staggered_steering_is_noise_free_target_snapshot(C, P, K, T, S, s0, k0):
    """A unit target at a bin centre on the steering grid gives the staggered
    snapshot v_{s0} = (sum h') a_{s0}, the same in every sub-window."""
    d = oracle.Dims(C, P, K, 8, T, 8, S)
    th = np.deg2rad(synth.steering_angle_deg(s0, S))
    cube = np.zeros((C, P, 8), np.complex128)
    cube[:, :, 5] = np.exp(2j * np.pi * 0.5 * np.sin(th) * np.arange(C))[:, None] * \
        np.exp(2j * np.pi * k0 / K * np.arange(P))[None, :]
    xs = oracle.doppler_staggered(d, cube)
    x = oracle.snapshot(oracle.staggered_dims(d), xs, k0, 5)
    v = oracle.default_steering_staggered(d)[s0]
    np.testing.assert_allclose(x, v, rtol=0, atol=1e-12 * np.abs(v).max())
    G = np.hanning(P - T + 1).sum()
    a = np.exp(2j * np.pi * 0.5 * np.sin(th) * np.arange(C))
    np.testing.assert_allclose(v, np.kron(np.full(T, G), a), rtol=0, atol=1e-12 * G)


def test_staggered_with_one_dof_is_the_adjacent_bin_path():
    """T = 1: one sub-window of all P pulses, the adjacent-bin transform and
    steering exactly."""
    d = dims(C=3, P=16, K=32, R=64, T=1, B=16, S=4)
    cube = crandn(3, 16, 64)
    np.testing.assert_array_equal(oracle.doppler_staggered(d, cube), oracle.doppler(d, cube))
    np.testing.assert_array_equal(oracle.default_steering_staggered(d), oracle.default_steering(d))
    np.testing.assert_array_equal(oracle.run(d, cube, staggered=True)["out"], oracle.run(d, cube)["out"])


def _amf_window_relative(C, P, K, R, T, B, S, cube, lf=1e-3):
    """The staggered STAP output written independently in numpy: sub-window t
    transformed relative to its own first pulse (numpy FFT), and the temporal
    steering that this phase reference needs, G exp(j 2 pi k t / K), which
    depends on the Doppler bin; np.linalg.solve for R^-1 v."""
    Ps = P - T + 1
    h = np.hanning(Ps)
    Y = np.stack([np.fft.fft(h[None, :, None] * cube[:, t:t + Ps, :], n=K, axis=1)
                  for t in range(T)])                       # [T][C][K][R]
    D, NB = C * T, R // B
    out = np.empty((S, K, R))
    ths = np.deg2rad(-90 + 180 * (np.arange(S) + 0.5) / S)
    A = np.exp(2j * np.pi * 0.5 * np.sin(ths)[:, None] * np.arange(C)[None, :])   # [S][C]
    for k in range(K):
        g = h.sum() * np.exp(2j * np.pi * k * np.arange(T) / K)
        V = np.stack([np.kron(g, A[s]) for s in range(S)])                         # [S][D]
        X = Y[:, :, k, :].reshape(D, R)                                            # rows t*C + c
        for b in range(NB):
            Xb = X[:, b * B:(b + 1) * B]
            Rm = Xb @ Xb.conj().T / B
            Rl = Rm + lf * np.trace(Rm).real / D * np.eye(D)
            U = np.linalg.solve(Rl, V.T)                                           # [D][S]
            q = np.einsum("ds,sd->s", U, V.conj()).real
            out[:, k, b * B:(b + 1) * B] = np.abs(U.conj().T @ Xb) ** 2 / q[:, None]
    return out


@pytest.mark.parametrize("C,P,K,R,T,B,S", [(3, 16, 16, 64, 3, 16, 4), (2, 12, 32, 48, 4, 16, 5)])
def test_staggered_run_equals_window_relative_form_with_doppler_dependent_steering(C, P, K, R, T, B, S):
    """Referencing each sub-window to its own first pulse multiplies bin k of
    sub-window t by exp(-j 2 pi k t / K) (a unitary diagonal change of basis)
    and moves that phase into a Doppler-dependent steering; the output power is
    the same."""
    d = oracle.Dims(C, P, K, R, T, B, S)
    cube = crandn(C, P, R)
    got = oracle.run(d, cube, staggered=True)["out"]
    ref = _amf_window_relative(C, P, K, R, T, B, S, cube)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * ref.max())


def test_staggered_run_is_composition_of_steps():
    d = dims(C=2, P=12, K=16, R=64, T=3, B=16, S=3)
    cube = crandn(2, 12, 64)
    res = oracle.run(d, cube, staggered=True, keep=True)
    e = oracle.staggered_dims(d)
    dop = oracle.doppler_staggered(d, cube)
    cov = oracle.covariance(e, dop)
    w, _, nf = oracle.weights(e, cov, oracle.default_steering_staggered(d))
    assert nf == 0
    np.testing.assert_array_equal(res["dop"], dop)
    np.testing.assert_array_equal(res["cov"], cov)
    np.testing.assert_array_equal(res["wts"], w)
    np.testing.assert_array_equal(res["out"], oracle.apply(e, dop, w))
    part = oracle.run(d, cube, r0=32, nr=16, staggered=True)
    np.testing.assert_array_equal(part["out"], res["out"][:, :, 32:48])


def test_staggered_small_workload_recovers_injected_target():
    """With staggered snapshots the small workload's target at (range 128,
    bin 24, steering 2) is still the strongest cell of its row, > 10 dB above
    the median."""
    spec = synth.small_cpi()
    d = oracle.Dims(*spec.dims())
    res = oracle.run(d, synth.make_cube(spec), staggered=True)
    P = res["out"]
    assert res["n_failed"] == 0
    assert int(np.argmax(P[2, 24])) == 128
    assert 10 * np.log10(P[2, 24, 128] / np.median(P)) > 10.0


# ------------------------------------------------ reduced-DOF front end ----
# N element channels combined into C channels by W[C][N]:
# y[c] = sum_n conj(W[c][n]) x[n]; default W: C contiguous subarrays.

def test_reduce_channels_is_the_conjugate_weighted_sum():
    W = crandn(3, 37)
    x = crandn(37, 5, 11)
    y = oracle.reduce_channels(W, x)
    np.testing.assert_allclose(y, np.einsum("cn,npr->cpr", W.conj(), x), rtol=0,
                               atol=1e-12 * np.abs(y).max())


def test_identity_front_end_is_the_plain_path():
    """W = I: the channels pass through, and the reduced steering is the default
    steering bit for bit."""
    d = dims(C=4, P=16, K=16, R=32, T=3, B=16, S=5)
    x = crandn(4, 16, 32)
    I4 = np.eye(4, dtype=np.complex128)
    np.testing.assert_array_equal(oracle.reduce_channels(I4, x), x)
    np.testing.assert_array_equal(oracle.reduced_steering(d, I4), oracle.default_steering(d))


@pytest.mark.parametrize("N,C,s0,k0", [(64, 4, 2, 5), (30, 3, 0, 11), (48, 8, 4, 0)])
def test_reduced_steering_is_the_noise_free_target_snapshot(N, C, s0, k0):
    """A unit plane wave on the steering grid at a bin centre, through the
    subarray front end, has snapshot v_{s0}."""
    P, K, T, S, R = 16, 16, 3, 5, 8
    d = oracle.Dims(C, P, K, R, T, 8, S)
    W = oracle.subarray_weights(N, C)
    th = np.deg2rad(synth.steering_angle_deg(s0, S))
    x = np.zeros((N, P, R), np.complex128)
    x[:, :, 3] = np.exp(2j * np.pi * 0.5 * np.sin(th) * np.arange(N))[:, None] * \
        np.exp(2j * np.pi * k0 / K * np.arange(P))[None, :]
    y = oracle.reduce_channels(W, x)
    snap = oracle.snapshot(d, oracle.doppler(d, y), k0, 3)
    v = oracle.reduced_steering(d, W)[s0]
    np.testing.assert_allclose(snap, v, rtol=0, atol=1e-12 * np.abs(v).max())


def test_subarray_weights_and_their_gain_closed_form():
    """Subarray c sums elements cM .. cM+M-1; its gain for spatial frequency f
    is the geometric series exp(j 2 pi f c M) (1 - e^{j 2 pi f M}) / (1 - e^{j 2 pi f})."""
    N, C, S = 40, 4, 6
    M = N // C
    W = oracle.subarray_weights(N, C)
    assert W.shape == (C, N) and np.all(W.imag == 0)
    for c in range(C):
        np.testing.assert_array_equal(W[c].real, (np.arange(N) // M == c).astype(float))
    d = oracle.Dims(C, 8, 8, 8, 1, 8, S)
    st = oracle.reduced_steering(d, W)             # T = 1: g_0 = sum h
    g0 = np.hanning(8).sum()
    for s in range(S):
        f = 0.5 * np.sin(np.deg2rad(synth.steering_angle_deg(s, S)))
        z = np.exp(2j * np.pi * f)
        b = z ** (np.arange(C) * M) * (1 - z ** M) / (1 - z)
        np.testing.assert_allclose(st[s], g0 * b, rtol=0, atol=1e-11 * np.abs(g0 * b).max())


def test_cube_window_equals_the_slice_of_the_whole_cube():
    """The input generator's range windows are the whole cube's slices, bit
    for bit (so windowed oracle runs see exactly the benchmark's input)."""
    for spec in (synth.small_cpi(),
                 synth.CPISpec(3, 20, 32, 96, 2, 32, 5, cnr_db=30.0,
                               targets=(synth.Target(50, 3, 1, 12.0),), seed=11)):
        whole = synth.make_cube(spec)
        for r0, nr in ((0, spec.training_block), (spec.n_range - 17, 17), (33, 40), (0, spec.n_range)):
            np.testing.assert_array_equal(synth.make_cube_window(spec, r0, nr), whole[:, :, r0:r0 + nr])
