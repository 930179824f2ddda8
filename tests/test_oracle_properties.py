"""Property checks of the oracle over random inputs (CPU; skipped where the
hypothesis package is missing): the cut-off's defining inequalities (Eq. 8-9),
reciprocity of the image method on coordinates exact in FP32, the log-Mel
frames following a shift of the signal by whole hops, and the paper's OLA
(Eq. 6) equal to the direct form (Eq. 3) for random shapes."""
import math

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = dict(max_examples=25, deadline=None, derandomize=True)


@settings(**SETTINGS)
@given(st.integers(1, 400), st.floats(0.0, 60.0), st.integers(0, 2 ** 31 - 1))
def test_cutoff_inequalities(n, eta, seed):
    rng = np.random.default_rng(seed)
    h = (rng.normal(0, 1, n) * np.exp(-np.arange(n) / max(1.0, n / 5))).astype(np.float32)
    L, peak, e_tot, e_kept = oracle.truncate(h, eta)
    p = h.astype(np.float64) ** 2
    assert 1 <= L <= n
    assert peak == pytest.approx(p.max(), rel=0, abs=0)
    if p.max() == 0:
        assert L == 1
        return
    p_th = p.max() * 10.0 ** (-eta / 10.0)
    # every sample from L on is below the threshold; n_c = L - 2 (when L < n) is not
    assert np.all(p[L:] < p_th)
    if L < n:
        assert L >= 2 and p[L - 2] >= p_th
    assert e_kept == pytest.approx(p[:L].sum(), rel=1e-12)
    assert e_tot == pytest.approx(p.sum(), rel=1e-12)


dyadic = st.integers(1, 31).map(lambda k: k / 8.0)


@settings(**SETTINGS)
@given(st.tuples(dyadic, dyadic, dyadic), st.tuples(dyadic, dyadic, dyadic), st.tuples(dyadic, dyadic, dyadic),
       st.floats(0.1, 0.95), st.integers(0, 3))
def test_image_method_reciprocity(room_k, src_k, mic_k, refl, order):
    room = tuple(4.0 + r for r in room_k)              # 4.125 .. 7.875 m
    src = tuple(min(s, r - 0.125) for s, r in zip(src_k, room))
    mic = tuple(min(m, r - 0.125) for m, r in zip(mic_k, room))
    if src == mic:
        return
    a, na = oracle.image_rir(room, src, mic, refl, 3000, order=order)
    b, nb = oracle.image_rir(room, mic, src, refl, 3000, order=order)
    assert na == nb
    np.testing.assert_array_equal(np.flatnonzero(a), np.flatnonzero(b))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


@settings(max_examples=10, deadline=None, derandomize=True)
@given(st.integers(0, 2 ** 31 - 1), st.integers(1, 5))
def test_log_mel_frames_follow_whole_hop_shifts(seed, k):
    rng = np.random.default_rng(seed)
    y = rng.normal(0, 0.1, 4000)
    shifted = np.concatenate([rng.normal(0, 0.1, 160 * k), y])
    a = oracle.log_mel(y, stack=1, stride=1)
    b = oracle.log_mel(shifted, stack=1, stride=1)
    np.testing.assert_allclose(b[k:k + a.shape[0]], a, rtol=0, atol=1e-9)


@settings(max_examples=15, deadline=None, derandomize=True)
@given(st.integers(1, 3000), st.integers(1, 3), st.integers(1, 2), st.integers(1, 300), st.integers(9, 12),
       st.integers(0, 2 ** 31 - 1))
def test_ola_equals_direct(nx, I, J, nh, log_n, seed):
    n_fft = 1 << log_n
    if nh > n_fft // 2:
        nh = n_fft // 2
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (I, nx))
    rirs = [rng.normal(0, 1, int(rng.integers(1, nh + 1))) for _ in range(I * J)]
    L = [len(r) for r in rirs]
    alpha = rng.uniform(0.2, 1.5, I)
    d = oracle.mix_direct(x, rirs, L, alpha)
    o = oracle.mix_ola(x, rirs, L, alpha, fft_n=n_fft)
    np.testing.assert_allclose(o, d, rtol=0, atol=1e-10 * max(1.0, np.abs(d).max()))
