"""Planted mistakes: each plausible error in the oracle must fail a pin.

A mutated copy of oracle.c is compiled into a temporary library and the pin
suite is run against it in a subprocess (ORACLE_LIB points the oracle's
loader at the mutant).  The pins are adequate only if every mutant fails.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, planted text)
MUTANTS = [
    ("eq9_keeps_one_less", "L = n_c + 2;", "L = n_c + 1;"),
    ("eq8_non_strict", "if (suffix < p_th) n_c = m;", "if (suffix <= p_th) n_c = m;"),
    ("eq7_amplitude_threshold", "double p_th = pmax * factor;", "double p_th = pmax * sqrt(factor);"),
    ("conv_drops_last_tap", "int64_t kmax = (n < Lij - 1) ? n : Lij - 1;\n            int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;\n            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];\n            yj[n]",
     "int64_t kmax = (n < Lij - 1) ? n : Lij - 2;\n            int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;\n            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];\n            yj[n]"),
    ("full_output_drops_first_tail_term",
     "int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;\n            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];\n            yj[n]",
     "int64_t kmin = (n - n_x + 2 > 0) ? n - n_x + 2 : 0;\n            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];\n            yj[n]"),
    ("full_dh_ignores_output_tail", "int64_t nend = (n_x + k < n_y) ? n_x + k : n_y;",
     "int64_t nend = (n_x < n_y) ? n_x : n_y;"),
    ("full_length_from_shortest_rir", "if (rir_len[r] > nh_max) nh_max = rir_len[r];",
     "if (r == lo->rir0[u] || rir_len[r] < nh_max) nh_max = rir_len[r];"),
    ("mix_ignores_gain", "yj[n] += alpha[i] * acc;", "yj[n] += acc;"),
    ("gain_snr_sign", "pow(10.0, -snr_db[i] / 10.0)", "pow(10.0, snr_db[i] / 10.0)"),
    ("gain_no_sqrt", "alpha[i] = sqrt(p0 / pi * pow(10.0, -snr_db[i] / 10.0));",
     "alpha[i] = p0 / pi * pow(10.0, -snr_db[i] / 10.0);"),
    ("dx_convolves_instead_of_correlates",
     "for (int64_t k = 0; k < Lij && m + k < n_y; ++k) acc += h[k] * gj[m + k];\n            dx_i[m]",
     "for (int64_t k = 0; k < Lij && m >= k; ++k) acc += h[k] * gj[m - k];\n            dx_i[m]"),
    ("window_dx_convolves",
     "for (int64_t k = 0; k < Lij && m + k < n_y; ++k) acc += h[k] * gj[m + k];\n            sum += acc;",
     "for (int64_t k = 0; k < Lij && m >= k; ++k) acc += h[k] * gj[m - k];\n            sum += acc;"),
    ("window_dh_drops_first_term", "for (int64_t n = k; n < nmax; ++n)", "for (int64_t n = k + 1; n < nmax; ++n)"),
    ("window_dh_ignores_cut", "        if (k < L_ij) {\n            int64_t nmax", "        if (1) {\n            int64_t nmax"),
    ("window_mix_ignores_gain", "sum += alpha[i] * acc;", "sum += acc;"),
    ("dh_transposed_operands", "acc += gj[n] * xi[n - k];", "acc += gj[n - k] * xi[n];"),
    ("dh_missing_gain", "dhij[k] = alpha[i] * acc;", "dhij[k] = acc;"),
    ("ola_hop_aliases", "int64_t hop = N - Lh + 1;", "int64_t hop = N - Lh + 2;"),
    ("ola_missing_normalisation", "yj[s + n] += alpha[i] * Br[n] / (double)N;",
     "yj[s + n] += alpha[i] * Br[n];"),
    ("fft_twiddle_sign", "double ang = sign * 2.0 * M_PI * (double)k / (double)len;",
     "double ang = -sign * 2.0 * M_PI * (double)k / (double)len;"),
]


# mistakes in the image-method RIR (Eq. 1), run against its own pin file
IMAGE_MUTANTS = [
    ("image_odd_parity_flipped", "(a % 2 == 0) ? (double)a", "(a % 2 != 0) ? (double)a"),
    ("image_f64_odd_coordinate", "(double)(a + 1) * len - s", "(double)a * len - s"),
    ("image_g_drops_axis", "im.g = abs(a) + abs(b) + abs(c);", "im.g = abs(a) + abs(b);"),
    ("image_delay_floor", "(int64_t)ceil(im.travel)", "(int64_t)floor(im.travel)"),
    ("image_delay_round", "(int64_t)ceil(im.travel)", "(int64_t)round(im.travel)"),
    ("image_amp_inverse_square", "(double)im.g) / d : 0.0;", "(double)im.g) / e2 : 0.0;"),
    ("image_fs_c0_swapped", "d * (double)fs / (double)c0;", "d * (double)c0 / (double)fs;"),
    ("image_loop_short", "for (int c = -order; c <= order; ++c) {\n                image_t im",
     "for (int c = -order; c < order; ++c) {\n                image_t im"),
    ("image_drops_last_sample", "if (im.delay < n_h) {", "if (im.delay < n_h - 1) {"),
    ("image_d2_misses_z", "e2 += ed * ed;", "if (k < 2) e2 += ed * ed;"),
]

# mistakes in the log-Mel front end, run against its own pin file
MEL_MUTANTS = [
    ("mel_symmetric_window", "cos(2.0 * M_PI * (double)n / (double)n_fft)",
     "cos(2.0 * M_PI * (double)n / (double)(n_fft - 1))"),
    ("mel_magnitude_not_power", "P[k] = re[k] * re[k] + im[k] * im[k];",
     "P[k] = sqrt(re[k] * re[k] + im[k] * im[k]);"),
    ("mel_scale_break_frequency", "2595.0 * log10(1.0 + f / 700.0)", "2595.0 * log10(1.0 + f / 1000.0)"),
    ("mel_edges_short_of_f_hi", "(double)(j + e) / (double)(n_mels + 1)", "(double)(j + e) / (double)(n_mels + 2)"),
    ("mel_falling_slope", "(edge[2] - f) / (edge[2] - edge[1])", "(edge[2] - f) / (edge[2] - edge[0])"),
    ("mel_floor_outside_log", "log(e + floor_)", "log(e) + floor_"),
    ("mel_stack_stride_confused", "F[(r * stride + s) * n_mels + j]", "F[(r * stack + s) * n_mels + j]"),
    ("mel_frame_start_shifted", "oracle_frame_power(y + t * hop, n_fft, P);",
     "oracle_frame_power(y + t * hop + 1, n_fft, P);"),
]

CASES = [(*m, "test_oracle_pins.py") for m in MUTANTS] + \
    [(*m, "test_oracle_image_pins.py") for m in IMAGE_MUTANTS] + \
    [(*m, "test_oracle_mel_pins.py") for m in MEL_MUTANTS]


@pytest.mark.parametrize("name,orig,planted,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted, pins):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / "oracle_mutant.c"
    mpath.write_text(src.replace(orig, planted))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-std=c11", "-D_DEFAULT_SOURCE", str(mpath), "-o", str(lib), "-lm"],
                   check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
