"""The oracle's pins must fail when a plausible mistake is planted in the oracle.

Each case copies the oracle source, changes one expression (a sign, an index, a
conjugate, a scale, a dropped term), compiles the copy on the CPU and runs the
pin suite against it in a subprocess; the suite must report a failure.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stap_oracle.c")

MUTANTS = {
    "dft_sign": ("double a = -2.0 * kPi * (double)m / (double)K;",
                 "double a = 2.0 * kPi * (double)m / (double)K;"),
    "snapshot_offset": ("int kk = ((k + t - T / 2) % K + K) % K;", "int kk = ((k + t) % K + K) % K;"),
    "covariance_scale": ("out[i] = Rm[i] / (double)B;", "out[i] = Rm[i];"),
    "covariance_conjugate": ("Rm[(size_t)i * D + j] += x[i] * conj(x[j]);",
                             "Rm[(size_t)i * D + j] += conj(x[i]) * x[j];"),
    "loading_dropped": ("A[(size_t)j * D + j] += delta;", "A[(size_t)j * D + j] += 0.0;"),
    "cholesky_conjugate": ("acc -= L[(size_t)i * D + k] * conj(L[(size_t)j * D + k]);",
                           "acc -= L[(size_t)i * D + k] * L[(size_t)j * D + k];"),
    "back_substitution_transpose": ("acc -= conj(L[(size_t)j * D + i]) * u[j];",
                                    "acc -= L[(size_t)j * D + i] * u[j];"),
    "normalisation_power": ("double scale = 1.0 / sqrt(q);", "double scale = 1.0 / q;"),
    "apply_conjugate": ("y += conj(W[(size_t)s * D + j]) * x[j];", "y += W[(size_t)s * D + j] * x[j];"),
    "hann_denominator": ("h[p] = 0.5 - 0.5 * cos(2.0 * kPi * (double)p / (double)(P - 1));",
                         "h[p] = 0.5 - 0.5 * cos(2.0 * kPi * (double)p / (double)P);"),
    "steering_sign": ("double fs = 0.5 * sin(theta);", "double fs = -0.5 * sin(theta);"),
    "steering_bin_offset": ("int m = t - T / 2;", "int m = t;"),
    "training_own_block": ("const cplx* lo = b > 0 ? cov_in + ((size_t)k * nb + b - 1) * DD : NULL;",
                           "const cplx* lo = b > 0 ? cov_in + ((size_t)k * nb + b) * DD : NULL;"),
    "training_mean_scale": ("if (lo && hi) o[e] = 0.5 * (lo[e] + hi[e]);",
                            "if (lo && hi) o[e] = lo[e] + hi[e];"),
    "window_includes_own_group": ("const int i = side == 0 ? j - guard - half + m : j + guard + 1 + m;",
                                  "const int i = side == 0 ? j - guard - half + m + 1 : j + guard + 1 + m;"),
    "window_mean_count": ("for (size_t e = 0; e < DD; ++e) o[e] /= (double)count;",
                          "for (size_t e = 0; e < DD; ++e) o[e] /= (double)(2 * half);"),
    "staggered_phase_reference": ("acc += h[p - t] * x * tw[((int64_t)p * k) % K];",
                                  "acc += h[p - t] * x * tw[((int64_t)(p - t) * k) % K];"),
    "staggered_window_length": ("const int Ps = P - T + 1;", "const int Ps = P - T;"),
    "staggered_steering_gain": ("for (int p = 0; p < Ps; ++p) G += h[p];",
                                "for (int p = 0; p < Ps; ++p) G += 1.0;"),
    "staggered_snapshot_order": ("dop[(((size_t)t * C + c) * K + k) * nr + rr] = acc;",
                                 "dop[(((size_t)c * T + t) * K + k) * nr + rr] = acc;"),
    "front_end_conjugate": ("acc += conj(W[(size_t)c * N + n]) * x[((size_t)n * P + p) * R + r];",
                            "acc += W[(size_t)c * N + n] * x[((size_t)n * P + p) * R + r];"),
    "front_end_steering_conjugate": (
        "for (int n = 0; n < N; ++n) acc += conj(W[(size_t)c * N + n]) * spatial_phase(s, S, n);",
        "for (int n = 0; n < N; ++n) acc += W[(size_t)c * N + n] * conj(spatial_phase(s, S, n));"),
    "subarray_membership": ("W[(size_t)c * N + n] = (n / M == c) ? 1.0 : 0.0;",
                            "W[(size_t)c * N + n] = (n % C == c) ? 1.0 : 0.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", str(mut), "-o", str(lib),
                    "-lm"], check=True)
    env = dict(os.environ, STAP_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
