"""Seeded synthetic radar cubes for the STAP path (inputs only).

This module holds the data model and nothing of the STAP method's arithmetic.
Both the CUDA path (through its tests and the benchmark) and the CPU oracle
take their inputs from here.

Random numbers: a counter-based SplitMix64 generator (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): sample ``i`` of
stream ``s`` under ``seed`` is ``mix(key(seed, s) + (i + 1) * 0x9E3779B97F4A7C15)``,
so every sample can be regenerated on its own.  Normal deviates come from the
Box-Muller transform in float64; the cube is rounded to complex64 once at the
end, and that complex64 cube is the canonical input.

Data model per CPI (cube[c][p][r], c < C channels, p < P pulses, r < R cells):

* noise: i.i.d. CN(0, 1) per sample (real and imaginary parts N(0, 1/2));
* clutter ridge: 64 patches at azimuths theta_i = -90 + 180 (i + 1/2)/64 deg,
  spatial frequency f_i = sin(theta_i)/2 and Doppler equal to it (beta = 1);
  per (patch, range cell) a CN(0, CNR/64) amplitude, constant over pulses and
  channels: sample += alpha_{i,r} exp(j 2 pi f_i c) exp(j 2 pi f_i p);
* targets: amplitude sqrt(SNR) exp(j phi) at one range cell r0, a Doppler-bin
  centre frequency k0/K and a steering-grid angle theta_{s0}:
  sample += a exp(j 2 pi f_{s0} c) exp(j 2 pi (k0/K) p).

CNR and SNR are per element per pulse (relative to the unit noise power).
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_NOISE = 0
STREAM_CLUTTER = 1
STREAM_TARGETS = 2
STREAM_BATCH_DIMS = 3

N_PATCH = 64


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int, sub: int = 0) -> np.uint64:
    a = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], np.uint64))
    b = _mix(a ^ np.array([(stream << 48) ^ (sub & 0xFFFFFFFFFFFF)], np.uint64))
    return b[0]


def uniform(seed: int, stream: int, idx, sub: int = 0) -> np.ndarray:
    """Uniform deviates in (0, 1) for the integer counters ``idx``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_key(seed, stream, sub) + (idx + np.uint64(1)) * _GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def complex_normal(seed: int, stream: int, idx, var: float = 1.0, sub: int = 0) -> np.ndarray:
    """CN(0, var) deviates (Box-Muller) for the counters ``idx`` (two uniforms each)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform(seed, stream, idx * np.uint64(2), sub)
    u2 = uniform(seed, stream, idx * np.uint64(2) + np.uint64(1), sub)
    rad = np.sqrt(-np.log(u1) * var)
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * (rad * np.sin(ang))


@dataclass(frozen=True)
class Target:
    r0: int          # range cell
    k0: int          # Doppler bin (normalised Doppler k0/K, wrapping above K/2)
    s0: int          # steering-grid index (angle theta_{s0})
    snr_db: float    # per element per pulse
    phase: float = 0.0


@dataclass(frozen=True)
class CPISpec:
    """Shape and content of one synthetic CPI."""
    n_chan: int
    n_pulses: int
    n_dop: int
    n_range: int
    tdof: int
    training_block: int
    n_steering: int
    cnr_db: Optional[float] = 40.0      # None: no clutter
    noise: bool = True
    targets: Tuple[Target, ...] = ()
    seed: int = 0
    sub: int = 0                          # CPI index inside a batch (substream)

    @property
    def D(self) -> int:
        return self.n_chan * self.tdof

    @property
    def NB(self) -> int:
        return self.n_range // self.training_block

    @property
    def cells(self) -> int:
        return self.n_dop * self.n_range

    def dims(self) -> Tuple[int, ...]:
        return (self.n_chan, self.n_pulses, self.n_dop, self.n_range, self.tdof,
                self.training_block, self.n_steering)


def steering_angle_deg(s: int, S: int) -> float:
    """The steering grid: uniform in angle over (-90, 90) degrees."""
    return -90.0 + 180.0 * (s + 0.5) / S


def patch_frequencies() -> np.ndarray:
    theta = np.deg2rad(-90.0 + 180.0 * (np.arange(N_PATCH) + 0.5) / N_PATCH)
    return 0.5 * np.sin(theta)


def random_targets(seed: int, n: int, R: int, K: int, S: int, snr_lo=0.0, snr_hi=15.0,
                   sub: int = 0) -> Tuple[Target, ...]:
    """n targets at seeded uniform (range, Doppler bin, steering index), SNR and phase."""
    u = uniform(seed, STREAM_TARGETS, np.arange(5 * n), sub).reshape(n, 5) if n else np.zeros((0, 5))
    out = []
    for j in range(n):
        out.append(Target(r0=int(u[j, 0] * R), k0=int(u[j, 1] * K), s0=int(u[j, 2] * S),
                          snr_db=float(snr_lo + (snr_hi - snr_lo) * u[j, 3]),
                          phase=float(2.0 * np.pi * u[j, 4])))
    return tuple(out)


def make_cube(spec: CPISpec, chan_chunk: int = 4) -> np.ndarray:
    """The complex64 cube [C][P][R] of ``spec`` (generated in float64, rounded once)."""
    C, P, R = spec.n_chan, spec.n_pulses, spec.n_range
    cube = np.empty((C, P, R), np.complex64)
    f = patch_frequencies()
    alpha = None
    if spec.cnr_db is not None:
        cnr = 10.0 ** (spec.cnr_db / 10.0)
        alpha = complex_normal(spec.seed, STREAM_CLUTTER, np.arange(N_PATCH * R, dtype=np.uint64),
                               cnr / N_PATCH, spec.sub).reshape(N_PATCH, R)
    dop_steer = np.exp(2j * np.pi * np.outer(np.arange(P), f))            # [P][patch]
    for c0 in range(0, C, chan_chunk):
        c1 = min(C, c0 + chan_chunk)
        blk = np.zeros((c1 - c0, P, R), np.complex128)
        if spec.noise:
            idx = np.arange(c0 * P * R, c1 * P * R, dtype=np.uint64)
            blk += complex_normal(spec.seed, STREAM_NOISE, idx, 1.0, spec.sub).reshape(c1 - c0, P, R)
        if alpha is not None:
            for c in range(c0, c1):
                sp = np.exp(2j * np.pi * f * c)                           # [patch]
                blk[c - c0] += (dop_steer * sp[None, :]) @ alpha
        cube[c0:c1] = blk
    if spec.targets:
        for t in spec.targets:
            th = np.deg2rad(steering_angle_deg(t.s0, spec.n_steering))
            fs = 0.5 * np.sin(th)
            amp = np.sqrt(10.0 ** (t.snr_db / 10.0)) * np.exp(1j * t.phase)
            sig = amp * np.exp(2j * np.pi * fs * np.arange(C))[:, None] * \
                np.exp(2j * np.pi * (t.k0 / spec.n_dop) * np.arange(P))[None, :]
            # add in float64 on top of the already-rounded value, then round again:
            # targets sit on single cells, so this equals generating them together
            # up to one extra rounding of those cells only.
            cube[:, :, t.r0] = (cube[:, :, t.r0].astype(np.complex128) + sig).astype(np.complex64)
    return cube


def make_cube_window(spec: CPISpec, r0: int, nr: int) -> np.ndarray:
    """Range cells [r0, r0 + nr) of ``make_cube(spec)``, bit for bit, without
    generating the rest of the cube (every sample's counters depend only on
    its own (channel, pulse, cell) and (patch, cell) indices)."""
    C, P, R = spec.n_chan, spec.n_pulses, spec.n_range
    if not (0 <= r0 and nr >= 0 and r0 + nr <= R):
        raise ValueError("window outside the range axis")
    cube = np.empty((C, P, nr), np.complex64)
    f = patch_frequencies()
    r = np.arange(r0, r0 + nr, dtype=np.uint64)
    alpha = None
    if spec.cnr_db is not None:
        cnr = 10.0 ** (spec.cnr_db / 10.0)
        idx = (np.arange(N_PATCH, dtype=np.uint64)[:, None] * np.uint64(R) + r[None, :]).ravel()
        alpha = complex_normal(spec.seed, STREAM_CLUTTER, idx, cnr / N_PATCH, spec.sub).reshape(N_PATCH, nr)
    dop_steer = np.exp(2j * np.pi * np.outer(np.arange(P), f))            # [P][patch]
    for c in range(C):
        blk = np.zeros((P, nr), np.complex128)
        if spec.noise:
            idx = (np.uint64(c * P * R) + np.arange(P, dtype=np.uint64)[:, None] * np.uint64(R) +
                   r[None, :]).ravel()
            blk += complex_normal(spec.seed, STREAM_NOISE, idx, 1.0, spec.sub).reshape(P, nr)
        if alpha is not None:
            sp = np.exp(2j * np.pi * f * c)
            blk += (dop_steer * sp[None, :]) @ alpha
        cube[c] = blk
    for t in spec.targets:
        if r0 <= t.r0 < r0 + nr:
            th = np.deg2rad(steering_angle_deg(t.s0, spec.n_steering))
            fs = 0.5 * np.sin(th)
            amp = np.sqrt(10.0 ** (t.snr_db / 10.0)) * np.exp(1j * t.phase)
            sig = amp * np.exp(2j * np.pi * fs * np.arange(C))[:, None] * \
                np.exp(2j * np.pi * (t.k0 / spec.n_dop) * np.arange(P))[None, :]
            j = t.r0 - r0
            cube[:, :, j] = (cube[:, :, j].astype(np.complex128) + sig).astype(np.complex64)
    return cube


# ----------------------------------------------------------------------------
# The workloads: a small single-CPI case, the standard single-CPI case, a
# mixed-precision case, a batch of uneven CPIs and a large single CPI.
# ----------------------------------------------------------------------------

def small_cpi() -> CPISpec:
    """C4 P32 K32 R256 T3 B32 S4, 30 dB CNR, one 10 dB target at (r 128, bin 24, steer 2)."""
    return CPISpec(4, 32, 32, 256, 3, 32, 4, cnr_db=30.0,
                   targets=(Target(128, 24, 2, 10.0, 0.0),), seed=1)


def standard_cpi() -> CPISpec:
    """C4 P128 K256 R4096 T3 B64 S16, 40 dB CNR, 8 targets at 0-15 dB SNR."""
    return CPISpec(4, 128, 256, 4096, 3, 64, 16, cnr_db=40.0,
                   targets=random_targets(2, 8, 4096, 256, 16), seed=2)


def mixed_cpi() -> CPISpec:
    """C16 P256 K256 R16384 T4 B128 S32, 40 dB CNR, 8 targets."""
    return CPISpec(16, 256, 256, 16384, 4, 128, 32, cnr_db=40.0,
                   targets=random_targets(3, 8, 16384, 256, 32), seed=3)


def mixed_small_cpi() -> CPISpec:
    """A quarter of the mixed workload (R = 4096) for profiling: C16 P256 K256 R4096 T4 B128 S32."""
    return CPISpec(16, 256, 256, 4096, 4, 128, 32, cnr_db=40.0,
                   targets=random_targets(3, 8, 4096, 256, 32), seed=3)


def large_cpi() -> CPISpec:
    """C32 P512 K512 R32768 T4 B256 S64, 40 dB CNR, 32 targets (about 4.3 GB)."""
    return CPISpec(32, 512, 512, 32768, 4, 256, 64, cnr_db=40.0,
                   targets=random_targets(5, 32, 32768, 512, 64), seed=5)


def large_small_cpi() -> CPISpec:
    """An eighth of the large workload (R = 4096, about 540 MB) for profiling:
    C32 P512 K512 R4096 T4 B256 S64."""
    return CPISpec(32, 512, 512, 4096, 4, 256, 64, cnr_db=40.0,
                   targets=random_targets(5, 8, 4096, 512, 64), seed=5)


def batch_cpis(n: int = 512, seed: int = 4) -> List[CPISpec]:
    """n uneven CPIs: C in {4,8,16}, T in {2,3,4}, P = K in {64,128,256},
    R = 64 * U{16..256}, B = 64, S in {8,16}, CNR uniform in 20-40 dB, 4 targets each."""
    u = uniform(seed, STREAM_BATCH_DIMS, np.arange(7 * n)).reshape(n, 7)
    out = []
    for i in range(n):
        C = (4, 8, 16)[int(u[i, 0] * 3)]
        T = (2, 3, 4)[int(u[i, 1] * 3)]
        P = (64, 128, 256)[int(u[i, 2] * 3)]
        R = 64 * (16 + int(u[i, 3] * 241))
        S = (8, 16)[int(u[i, 4] * 2)]
        cnr = 20.0 + 20.0 * float(u[i, 5])
        out.append(CPISpec(C, P, P, R, T, 64, S, cnr_db=cnr,
                           targets=random_targets(seed, 4, R, P, S, sub=i + 1),
                           seed=seed, sub=i + 1))
    return out


def paper_cube_elements() -> CPISpec:
    """The element cube of the paper's STAP data shape (Sec. 5.3: 1000 channels,
    100 pulses, 30000 samples per pulse; about 24 GB as complex64), as elements
    of a half-wavelength line array: 40 dB CNR per element, 8 targets.  Its
    K, T, B, S (128, 3, 100, 16) are the chain's after a front end that
    reduces the 1000 elements to PAPER_CUBE_CHANNELS channels."""
    return CPISpec(1000, 100, 128, 30000, 3, 100, 16, cnr_db=40.0,
                   targets=random_targets(6, 8, 30000, 128, 16), seed=6)


PAPER_CUBE_CHANNELS = 4     # contiguous subarrays of 250 elements


def paper_cube_small_elements() -> CPISpec:
    """The paper cube with a tenth of its range (R = 3000, about 2.4 GB), for
    profiles of the front end."""
    return CPISpec(1000, 100, 128, 3000, 3, 100, 16, cnr_db=40.0,
                   targets=random_targets(6, 8, 3000, 128, 16), seed=6)


ELEMENT_WORKLOADS = {
    "paper_cube": paper_cube_elements,
    "paper_cube_small": paper_cube_small_elements,
}


WORKLOADS = {
    "small": small_cpi,
    "standard": standard_cpi,
    "mixed": mixed_cpi,
    "mixed_small": mixed_small_cpi,
    "large": large_cpi,
    "large_small": large_small_cpi,
}


# ----------------------------------------------------------------------------
# The same recipe evaluated on a CUDA device (for cubes of several GB).  The
# counters and SplitMix64 mixing are bit-identical to the numpy version; the
# Box-Muller transcendentals and the clutter matrix product may differ in the
# last bits, so tests always hand the oracle the device cube copied back.
# ----------------------------------------------------------------------------

def _signed(x: int) -> int:
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def _mix_t(z):
    z = z ^ ((z >> 30) & ((1 << 34) - 1))          # logical shifts on int64 bit patterns
    z = z * _signed(0xBF58476D1CE4E5B9)
    z = z ^ ((z >> 27) & ((1 << 37) - 1))
    z = z * _signed(0x94D049BB133111EB)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def _uniform_t(seed, stream, idx, sub=0):
    import torch
    key = _signed(int(_key(seed, stream, sub)))
    z = _mix_t(key + (idx + 1) * _signed(0x9E3779B97F4A7C15))
    return (((z >> 11) & ((1 << 53) - 1)).to(torch.float64) + 0.5) * (1.0 / 9007199254740992.0)


def _complex_normal_t(seed, stream, idx, var, sub=0):
    import torch
    u1 = _uniform_t(seed, stream, idx * 2, sub)
    u2 = _uniform_t(seed, stream, idx * 2 + 1, sub)
    rad = torch.sqrt(-torch.log(u1) * var)
    ang = (2.0 * np.pi) * u2
    return torch.complex(rad * torch.cos(ang), rad * torch.sin(ang))


def make_cube_torch(spec: CPISpec, device="cuda"):
    """The complex64 cube of ``spec`` computed on ``device`` (torch tensor)."""
    import torch
    C, P, R = spec.n_chan, spec.n_pulses, spec.n_range
    dev = torch.device(device)
    cube = torch.empty((C, P, R), dtype=torch.complex64, device=dev)
    f = torch.from_numpy(patch_frequencies()).to(dev)
    alpha = None
    if spec.cnr_db is not None:
        cnr = 10.0 ** (spec.cnr_db / 10.0)
        idx = torch.arange(N_PATCH * R, dtype=torch.int64, device=dev)
        alpha = _complex_normal_t(spec.seed, STREAM_CLUTTER, idx, cnr / N_PATCH, spec.sub).reshape(N_PATCH, R)
    p = torch.arange(P, dtype=torch.float64, device=dev)
    dop_steer = torch.exp(torch.complex(torch.zeros_like(p[:, None] * f[None, :]),
                                        2.0 * np.pi * p[:, None] * f[None, :]))   # [P][patch]
    base = torch.arange(P * R, dtype=torch.int64, device=dev)
    for c in range(C):
        blk = torch.zeros((P, R), dtype=torch.complex128, device=dev)
        if spec.noise:
            blk += _complex_normal_t(spec.seed, STREAM_NOISE, base + c * P * R, 1.0, spec.sub).reshape(P, R)
        if alpha is not None:
            ph = 2.0 * np.pi * f * c
            sp = torch.complex(torch.cos(ph), torch.sin(ph))
            blk += (dop_steer * sp[None, :]) @ alpha
        cube[c] = blk.to(torch.complex64)
    for t in spec.targets:
        th = np.deg2rad(steering_angle_deg(t.s0, spec.n_steering))
        fs = 0.5 * np.sin(th)
        amp = np.sqrt(10.0 ** (t.snr_db / 10.0)) * np.exp(1j * t.phase)
        sig = amp * np.exp(2j * np.pi * fs * np.arange(C))[:, None] * \
            np.exp(2j * np.pi * (t.k0 / spec.n_dop) * np.arange(P))[None, :]
        col = cube[:, :, t.r0].to(torch.complex128) + torch.from_numpy(sig).to(dev)
        cube[:, :, t.r0] = col.to(torch.complex64)
    return cube
