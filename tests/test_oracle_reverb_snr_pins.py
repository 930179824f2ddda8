"""Pins of the oracle's gains from SNRs measured on the reverberant signal at a
reference microphone: the requested SNR is met between the target's and each
noise source's contribution to that microphone's mixed output, the gains do
not depend on the other microphones, and with unit-impulse RIRs they are the
dry-signal gains."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth


def batch(seed=5):
    b = synth.make_batch(seed, [1500, 2300], [3, 2], synth.linear_pair_array(), (0.05, 0.1), n_taps=400)
    return synth.trim_rirs(b, seed + 1)


@pytest.mark.parametrize("ref", [0, 1])
def test_requested_snr_is_met_at_the_reference_mic(ref):
    b = batch()
    alpha, _ = oracle.reverberant_gains(b, eta_db=20.0, ref_mic=ref)
    si, J = b.src_index(), b.num_mics
    yo = b.y_offsets()
    for u in range(b.num_utts):
        nx = int(b.num_samples[u])
        powers = []
        for i in range(int(b.num_sources[u])):
            a = np.zeros(int(si[-1]))
            a[si[u] + i] = alpha[si[u] + i]
            y = oracle.forward(b, 20.0, alpha=a)["y"]         # that source alone, scaled
            yj = y[yo[u] + ref * nx:yo[u] + (ref + 1) * nx]
            powers.append(np.mean(yj ** 2))
        for i in range(1, len(powers)):
            assert 10 * math.log10(powers[0] / powers[i]) == pytest.approx(b.snr_db[si[u] + i], abs=1e-9)


def test_other_mics_do_not_matter():
    b = batch(7)
    a0, _ = oracle.reverberant_gains(b, ref_mic=0)
    ro, J = b.rir_offsets(), b.num_mics
    rir = b.rir.copy()
    for r in range(b.num_rirs):
        if r % J == 1:
            rir[ro[r]:ro[r + 1]] *= 3.0
    import dataclasses
    a1, _ = oracle.reverberant_gains(dataclasses.replace(b, rir=rir), ref_mic=0)
    np.testing.assert_array_equal(a0, a1)


def test_unit_impulse_rirs_give_the_dry_gains():
    b = batch(9)
    import dataclasses
    rir = np.zeros_like(b.rir)
    rir[b.rir_offsets()[:-1]] = 1.0
    d = dataclasses.replace(b, rir=rir)
    a, _ = oracle.reverberant_gains(d, eta_db=20.0, ref_mic=1)
    dry = oracle.forward(b, 20.0)["alpha"]
    np.testing.assert_allclose(a, dry, rtol=1e-12)
