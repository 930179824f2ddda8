"""Pins of the oracle's log-Mel front end (Sec. 3 features) against facts that
do not come from the oracle itself:

* the HTK Mel scale maps 1000 Hz to 1000 Mel (the property it is built on) and
  700 Hz to 2595 log10 2;
* adjacent triangular filters sum to one between the first and the last
  centre, every filter is zero outside [f_lo, f_hi], and the band edges reach
  the bins next to f_lo and f_hi;
* the Hann-windowed power spectrum of a tone on a bin is three lines of known
  height (N A / 4 and N A / 8 in amplitude); Parseval; numpy's rfft;
* a constant signal has no energy above 125 Hz, so every feature is ln(floor);
* scaling the signal shifts the features by 2 ln(scale);
* frame count, frame positions and the stacked layout, by brute force.
"""
import math

import numpy as np
import pytest

import oracle

N_FFT, HOP, FS = 512, 160, 16000.0


def test_htk_mel_scale_anchors():
    assert oracle.hz_to_mel(1000.0) == pytest.approx(1000.0, abs=0.05)
    assert oracle.hz_to_mel(700.0) == pytest.approx(2595.0 * math.log10(2.0), rel=1e-15)
    assert oracle.hz_to_mel(0.0) == 0.0
    for f in (125.0, 1000.0, 7500.0):
        assert oracle.mel_to_hz(oracle.hz_to_mel(f)) == pytest.approx(f, rel=1e-12)


def test_filters_partition_unity_and_stay_in_band():
    W = oracle.mel_filters()
    assert W.shape == (128, 257)
    f = np.arange(257) * FS / N_FFT
    assert np.all(W >= 0) and np.all(W <= 1.0 + 1e-12)
    # zero outside [125, 7500] Hz; the outermost bins inside the band carry weight
    assert not W[:, (f <= 125.0) | (f >= 7500.0)].any()
    inside = np.flatnonzero(W.sum(0) > 0)
    assert f[inside[-1]] == 7468.75 and f[inside[0]] < 160.0
    # between the peaks of the first and the last non-empty filter the triangles sum to
    # one (the lowest filters are narrower than a bin: some hold no bin at all)
    used = np.flatnonzero(W.sum(1) > 0)
    assert used.size >= 120 and used[-1] == 127
    c0 = f[np.argmax(W[used[0]])]
    c1 = f[np.argmax(W[-1])]
    mid = (f > c0) & (f < c1)
    np.testing.assert_allclose(W[:, mid].sum(0), 1.0, rtol=0, atol=1e-12)
    # each filter rises then falls (one peak, no holes)
    for j in range(128):
        nz = np.flatnonzero(W[j])
        if nz.size:
            assert np.all(np.diff(nz) == 1)
            k = int(np.argmax(W[j, nz]))
            assert np.all(np.diff(W[j, nz[:k + 1]]) > 0) and np.all(np.diff(W[j, nz[k:]]) < 0)


@pytest.mark.parametrize("k0,amp,phase", [(64, 0.3, 0.0), (17, 1.0, 0.7), (200, 0.05, -1.3)])
def test_hann_tone_spectrum_closed_form(k0, amp, phase):
    n = np.arange(N_FFT)
    x = amp * np.cos(2 * np.pi * k0 * n / N_FFT + phase)
    P = oracle.frame_power(x)
    want = np.zeros(N_FFT // 2 + 1)
    want[k0] = (N_FFT * amp / 4) ** 2
    want[k0 - 1] = want[k0 + 1] = (N_FFT * amp / 8) ** 2
    np.testing.assert_allclose(P, want, rtol=1e-10, atol=1e-18 * N_FFT ** 2 + 1e-20)


def test_frame_power_parseval_and_rfft():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 0.2, N_FFT)
    P = oracle.frame_power(x)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(N_FFT) / N_FFT)
    xw = w * x
    assert (P[0] + 2 * P[1:-1].sum() + P[-1]) / N_FFT == pytest.approx(np.sum(xw ** 2), rel=1e-12)
    np.testing.assert_allclose(P, np.abs(np.fft.rfft(xw)) ** 2, rtol=1e-10, atol=1e-12)


def test_constant_signal_has_no_band_energy():
    f = oracle.log_mel(np.full(4000, 0.4))
    assert f.shape == (7, 512)
    np.testing.assert_allclose(f, math.log(1e-6), rtol=0, atol=1e-9)


def test_scaling_shifts_features():
    rng = np.random.default_rng(4)
    y = rng.normal(0, 0.1, 8000)
    a = oracle.log_mel(y, floor=0.0)
    b = oracle.log_mel(3.0 * y, floor=0.0)
    band = np.isfinite(a)          # empty filters give ln 0
    assert band.mean() > 0.9
    np.testing.assert_allclose(b[band] - a[band], 2 * math.log(3.0), rtol=0, atol=1e-9)


@pytest.mark.parametrize("n", [0, 511, 512, 671, 672, 1000, 1150, 1151, 16000, 16001])
def test_frame_and_row_counts(n):
    frames = sum(1 for t in range(n) if t * HOP + N_FFT <= n)
    rows = sum(1 for r in range(frames) if 3 * r + 3 < frames)
    assert oracle.log_mel_rows(n) == rows
    assert oracle.log_mel(np.zeros(n)).shape == (rows, 512)


def test_stacked_layout_and_frame_positions():
    rng = np.random.default_rng(5)
    y = rng.normal(0, 0.1, 3000)
    one = oracle.log_mel(y, stack=1, stride=1)          # one row per frame
    assert one.shape == ((3000 - 512) // 160 + 1, 128)
    st = oracle.log_mel(y)
    for r in range(st.shape[0]):
        for s in range(4):
            np.testing.assert_array_equal(st[r, s * 128:(s + 1) * 128], one[3 * r + s])
    # frame t sees samples [160 t, 160 t + 512) only
    t = 5
    z = y.copy()
    z[t * 160 - 1] += 1.0        # last sample before frame t: frames t and later unchanged
    z[t * 160 + 512] += 1.0      # first sample after frame t
    two = oracle.log_mel(z, stack=1, stride=1)
    np.testing.assert_array_equal(two[t], one[t])
    z = y.copy()
    z[t * 160 + 256] += 1.0   # (sample 0 of a frame has Hann weight 0)
    assert not np.array_equal(oracle.log_mel(z, stack=1, stride=1)[t], one[t])


def test_batch_matches_single_calls():
    rng = np.random.default_rng(6)
    ny = np.array([3000, 400, 5000, 1151], np.int64)
    J = 2
    y = rng.normal(0, 0.1, int(ny.sum()) * J)
    for ch in (0, 1):
        out, off = oracle.log_mel_batch(y, ny, J, channel=ch)
        yo = np.concatenate([[0], np.cumsum(ny * J)])
        for u in range(4):
            want = oracle.log_mel(y[yo[u] + ch * ny[u]:yo[u] + (ch + 1) * ny[u]])
            np.testing.assert_array_equal(out[off[u]:off[u + 1]], want)
