"""RIRs longer than one block of the largest FFT size reaches, without a
cut-off: uniformly partitioned convolution (virtual sources delayed by whole
parts, each with one part of the RIRs) against the FP64 oracle's direct
convolution with the whole RIRs.  Tolerances as for the per-source path."""
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


def check_channels(y, ref, b):
    yo = b.y_offsets()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(b.num_mics):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            r = ref[s]
            if not np.any(r):
                assert not np.any(y[s])
                continue
            assert rel_l2(y[s], r) <= REL, f"y u={u} j={j}"
            assert np.max(np.abs(y[s] - r)) <= REL * np.max(np.abs(r)), f"y u={u} j={j} max abs"


@pytest.mark.parametrize("gain_mode,fft_sizes", [(1, None), (0, None), (1, [8192]), (0, [4096, 16384])])
def test_partitioned_forward_and_backward_match_oracle(gain_mode, fft_sizes):
    from paper_1712_03439_gb300 import Plan
    b = synth.trim_rirs(synth.make_batch(201, [1, 700, 20011, 33333], [1, 2, 3, 2], synth.linear_pair_array(),
                                         (0.9, 1.2)), 202, min_frac=0.5)
    assert b.rir_len.max() > 12289
    plan = Plan.for_batch(b, eta_db=math.inf, gain_mode=gain_mode, fft_sizes=fft_sizes)
    S = int(b.num_sources.sum())
    x, rir = dev(b.x), dev(b.rir)
    gains = dev(np.linspace(0.6, 1.3, S)) if gain_mode == 1 else torch.empty(S, device="cuda")
    y = torch.full((plan.y_size,), float("nan"), device="cuda")
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    for _ in range(2):                       # the second call replays the captured graph
        plan.filter_mix(x, rir, gains, y, snr_db=dev(b.snr_db) if gain_mode == 0 else None, trunc_len=tl)
    plan.sync_status()
    np.testing.assert_array_equal(tl.cpu().numpy(), b.rir_len)
    alpha = gains.cpu().numpy().astype(np.float64)
    if gain_mode == 0:
        np.testing.assert_allclose(alpha, oracle.forward(b, math.inf)["alpha"], rtol=REL)
    ref = oracle.forward(b, math.inf, alpha=alpha)
    check_channels(y.cpu().numpy(), ref["y"], b)
    gy = synth.grad_like(203, b.y_size)
    gx, gr, gg = torch.empty_like(x), torch.full_like(rir, float("nan")), torch.empty(S, device="cuda")
    plan.filter_mix_backward(dev(gy), x, gains, gx, gr, gg)
    plan.sync_status()
    bw = oracle.backward(b, b.rir_len.astype(np.int64), alpha, gy.astype(np.float64))
    grads_close(b, bw, b.rir_len, dx=gx.cpu().numpy(), dh=gr.cpu().numpy(), dalpha=gg.cpu().numpy())
    q = plan.query()
    assert np.all(q["log2_n"] > 0)


@pytest.mark.parametrize("kw", [dict(output_mode=1), dict(gain_mode=2), dict(gain_mode=3)])
def test_partitioned_unsupported_combinations(kw):
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(211, [5000], [2], synth.linear_pair_array(), (1.0, 1.0))
    kw = dict(dict(gain_mode=1), **kw)
    with pytest.raises(RsimError) as e:
        Plan.for_batch(b, eta_db=math.inf, **kw)
    assert e.value.status == 2


def test_too_many_parts_is_unsupported():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(212, [5000], [6], synth.linear_pair_array(), (1.2, 1.2))   # 6 x 3 parts > 16
    with pytest.raises(RsimError) as e:
        Plan.for_batch(b, eta_db=math.inf, gain_mode=1)
    assert e.value.status == 2
