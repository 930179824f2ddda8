"""Gains from SNRs measured on the reverberant signal at a reference
microphone (gain mode 3): CUDA path vs the FP64 oracle.  Gains within a
relative 1e-5 (they come from FP32 sums of squares of the FP32 filtered
sources); the mix with those gains and its adjoint with the tolerances of the
per-source path (per channel or vector relative L2 <= 1e-5)."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth
from parity_checks import close_vec, grads_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, r):
    return np.linalg.norm(np.asarray(a, np.float64) - r) / max(np.linalg.norm(r), 1e-30)


@pytest.mark.parametrize("J,ref,eta,graphs", [(2, 0, 20.0, True), (2, 1, 20.0, False), (3, 2, math.inf, True)])
def test_reverberant_gains_and_mix_match_oracle(J, ref, eta, graphs):
    from paper_1712_03439_gb300 import Plan
    mics = synth.linear_pair_array() if J == 2 else synth.circular_array(J, 0.05)
    b = synth.make_batch(100 + J + ref, [3000, 20011, 47000, 9000], [3, 2, 4, 1], mics, (0.1, 0.25))
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=3, snr_ref_mic=ref, graphs=graphs)
    x, rir, snr = dev(b.x), dev(b.rir), dev(b.snr_db)
    gains = torch.empty(plan.S, device="cuda")
    y = torch.empty(plan.y_size, device="cuda")
    for _ in range(2):                       # the second call replays the captured graph
        plan.filter_mix(x, rir, gains, y, snr_db=snr)
    plan.sync_status()
    alpha, _ = oracle.reverberant_gains(b, eta_db=eta, ref_mic=ref)
    np.testing.assert_allclose(gains.cpu().numpy(), alpha, rtol=REL, atol=0)
    ref_y = oracle.forward(b, eta, alpha=alpha)["y"]
    yo = b.y_offsets()
    yg = y.cpu().numpy()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(J):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            close_vec(yg[s], ref_y[s], f"y u={u} j={j}")
    # the adjoint treats the gains as inputs (as in gain mode 0)
    gy = synth.grad_like(7, b.y_size)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty(plan.S, device="cuda")
    plan.filter_mix_backward(dev(gy), x, gains, gx, gr, gg)
    plan.sync_status()
    L = oracle.truncate_batch(b, eta)["L"]
    bw = oracle.backward(b, L, gains.cpu().numpy().astype(np.float64), gy.astype(np.float64))
    grads_close(b, bw, L, dx=gx.cpu().numpy(), dh=gr.cpu().numpy(), dalpha=gg.cpu().numpy())


def test_reference_mic_out_of_range_is_rejected():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(5, [3000], [2], synth.linear_pair_array(), (0.1, 0.2))
    with pytest.raises(RsimError):
        Plan.for_batch(b, gain_mode=3, snr_ref_mic=2)


def test_silent_reverberant_source_is_reported():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(6, [4000], [2], synth.linear_pair_array(), (0.1, 0.2))
    ro, ri = b.rir_offsets(), b.rir_index()
    r = int(ri[0]) + 1 * b.num_mics + 1          # noise source 1 to microphone 1
    b.rir[ro[r]:ro[r + 1]] = 0.0
    plan = Plan.for_batch(b, gain_mode=3, snr_ref_mic=1)
    gains, y = torch.empty(plan.S, device="cuda"), torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(dev(b.x), dev(b.rir), gains, y, snr_db=dev(b.snr_db))
    with pytest.raises(RsimError) as e:
        plan.sync_status()
    assert e.value.status == 1
