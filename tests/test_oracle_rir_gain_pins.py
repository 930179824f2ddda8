"""Pins of the oracle's per-(source, microphone) gains (Eq. 2's alpha_ij):
with alpha_ij = alpha_i it is the per-source mix and its adjoint exactly;
the output is linear in the gains; central finite differences in FP64 give
every dalpha_ij; the adjoint identity <dy, g> = <dalpha, delta alpha> holds."""
import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth


def small_batch(seed=11):
    b = synth.make_batch(seed, [900, 1300], [2, 3], synth.linear_pair_array(), (0.05, 0.08), n_taps=300)
    return synth.trim_rirs(b, seed + 1)


def test_per_source_gains_are_the_special_case():
    b = small_batch()
    J = b.num_mics
    alpha_s = np.array([1.0, 0.4, 1.0, 0.7, 0.2])
    alpha_r = np.repeat(alpha_s, J)
    ref = oracle.forward(b, 20.0, alpha=alpha_s)
    got = oracle.forward_rir_gains(b, alpha_r, 20.0)
    np.testing.assert_array_equal(got["L"], ref["L"])
    np.testing.assert_allclose(got["y"], ref["y"], rtol=1e-13, atol=1e-15)
    g = synth.grad_like(3, ref["y"].shape[0]).astype(np.float64)
    rb = oracle.backward(b, ref["L"], alpha_s, g)
    gb = oracle.backward_rir_gains(b, ref["L"], alpha_r, g)
    np.testing.assert_allclose(gb["dx"], rb["dx"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gb["dh"], rb["dh"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gb["dalpha"].reshape(-1, J).sum(1), rb["dalpha"], rtol=1e-10, atol=1e-12)


def test_linear_in_the_gains():
    b = small_batch(12)
    rng = np.random.default_rng(1)
    a1, a2 = rng.uniform(-1, 1, b.num_rirs), rng.uniform(-1, 1, b.num_rirs)
    y1 = oracle.forward_rir_gains(b, a1)["y"]
    y2 = oracle.forward_rir_gains(b, a2)["y"]
    y12 = oracle.forward_rir_gains(b, 2.0 * a1 - 0.5 * a2)["y"]
    np.testing.assert_allclose(y12, 2.0 * y1 - 0.5 * y2, rtol=1e-12, atol=1e-13)


def test_finite_differences_and_adjoint_identity():
    b = small_batch(13)
    rng = np.random.default_rng(2)
    a = rng.uniform(0.2, 1.0, b.num_rirs)
    fwd = oracle.forward_rir_gains(b, a, eta_db=float("inf"))
    L = fwd["L"]
    t = rng.normal(0, 0.1, fwd["y"].shape[0])

    def loss(al):
        y = oracle.forward_rir_gains(b, al, eta_db=float("inf"))["y"]
        return 0.5 * np.sum((y - t) ** 2)
    g = fwd["y"] - t
    bw = oracle.backward_rir_gains(b, L, a, g)
    for r in range(b.num_rirs):
        e = np.zeros_like(a)
        e[r] = 1e-4
        fd = (loss(a + e) - loss(a - e)) / 2e-4
        assert bw["dalpha"][r] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # <d y / d alpha . delta, g> = <dalpha, delta>
    delta = rng.normal(0, 1, b.num_rirs)
    dy = oracle.forward_rir_gains(b, delta, eta_db=float("inf"))["y"]   # y is linear in alpha
    assert np.dot(dy, g) == pytest.approx(np.dot(bw["dalpha"], delta), rel=1e-10)
