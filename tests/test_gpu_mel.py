"""Log-Mel front end (Sec. 3 features): CUDA path vs the FP64 oracle.

The frame and row bookkeeping is integer work and must match exactly (row
counts, which frame lands in which row and slot).  Values are compared in the
energy domain, where FP32 errors scale with the frame's strongest band: per
stacked frame, every filter energy E = exp(v) - floor within 1e-5 of the
frame's largest energy, and the log features of the bands within 30 dB of it
within 1e-4 (an FP32 FFT of 512 points and FP32 filter edges sit near 3e-7
and 1e-6 there).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 1e-5
V_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def check_features(got, want, n_mels, floor, what):
    assert got.shape == want.shape, what
    assert np.all(np.isfinite(got)), what
    g = got.reshape(-1, n_mels).astype(np.float64)
    w = want.reshape(-1, n_mels)
    eg, ew = np.exp(g) - floor, np.exp(w) - floor
    scale = ew.max(axis=1, keepdims=True)
    assert np.all(np.abs(eg - ew) <= E_TOL * scale + 1e-3 * floor), what
    strong = ew >= 1e-3 * scale
    assert np.all(np.abs(g - w)[strong] <= V_TOL), what


def mixed_output(plan, seed):
    """A mixed-output stand-in of the plan's layout: speech-like signal per
    microphone channel of every utterance."""
    rng = np.random.default_rng(seed)
    parts = []
    for n in plan.num_out:
        for _ in range(plan.num_mics):
            parts.append(synth.speech_like(rng, int(n)) if n > 0 else np.zeros(0, np.float32))
    return np.concatenate(parts).astype(np.float32)


def small_plan(lengths, J=2, seed=3):
    from paper_1712_03439_gb300 import Plan
    b = synth.make_batch(seed, lengths, [1] * len(lengths), synth.circular_array(J, 0.05) if J > 2
                         else synth.linear_pair_array() if J == 2 else np.zeros((1, 2)), (0.1, 0.2))
    return Plan.for_batch(b, eta_db=20.0, gain_mode=1)


@pytest.mark.parametrize("kw", [
    dict(),                                                       # the paper's features
    dict(stack=1, stride=1),                                      # one row per frame
    dict(hop=100, n_mels=40, f_lo=0.0, f_hi=8000.0, channel=1),   # other band and hop, mic 1
    dict(hop=256, n_mels=1, stack=2, stride=5),
    dict(n_mels=97, log_floor=1e-3, stack=3, stride=2, fs=8000.0, f_lo=50.0, f_hi=3900.0),
])
def test_log_mel_matches_oracle(kw):
    lengths = [300, 511, 512, 671, 1151, 1152, 16000, 40001, 5123]
    plan = small_plan(lengths)
    y = mixed_output(plan, 7)
    feats = plan.log_mel(torch.from_numpy(y).cuda(), **kw)
    torch.cuda.synchronize()
    p = dict(oracle.MEL_DEFAULTS)
    p.update({k: v for k, v in kw.items() if k in p})
    if "log_floor" in kw:
        p["floor"] = kw["log_floor"]
    want, off = oracle.log_mel_batch(y, plan.num_out, plan.num_mics, channel=kw.get("channel", 0),
                                     **{k: v for k, v in p.items()})
    rows, total = plan.log_mel_rows(**kw)
    np.testing.assert_array_equal(np.concatenate([[0], np.cumsum(rows)]), off)
    assert feats.shape == (total, p["stack"] * p["n_mels"])
    check_features(feats.cpu().numpy(), want, p["n_mels"], p["floor"], str(kw))


def test_utterances_without_rows_write_nothing():
    plan = small_plan([100, 511, 600, 900])     # 0, 0, 1 and 3 frames: no row needs 4
    rows, total = plan.log_mel_rows()
    assert rows.tolist() == [0, 0, 0, 0] and total == 0
    y = torch.from_numpy(mixed_output(plan, 8)).cuda()
    sentinel = torch.full((1, 512), 7.0, device="cuda")
    plan.log_mel(y, feats=sentinel[:0])
    torch.cuda.synchronize()
    assert torch.all(sentinel == 7.0)


def test_home_workload_mixed_output_sampled():
    """The benchmark's launch: features of microphone 0 of the home-256 mix's
    real output, sampled utterances against the oracle."""
    from paper_1712_03439_gb300 import Plan
    b = synth.config_home()
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=0)
    x, rir, snr = (torch.from_numpy(a).cuda() for a in (b.x, b.rir, b.snr_db))
    gains = torch.empty(plan.S, device="cuda")
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(x, rir, gains, y, snr_db=snr)
    feats = plan.log_mel(y)
    torch.cuda.synchronize()
    rows, total = plan.log_mel_rows()
    off = np.concatenate([[0], np.cumsum(rows)])
    yh = y.cpu().numpy().astype(np.float64)
    f = feats.cpu().numpy()
    yo = b.y_offsets()
    for u in (0, 77, 128, 255):
        n = int(b.num_samples[u])
        want = oracle.log_mel(yh[yo[u]:yo[u] + n])
        check_features(f[off[u]:off[u + 1]], want, 128, 1e-6, f"utterance {u}")


def test_bad_descriptions_are_rejected():
    from paper_1712_03439_gb300._lib import RsimError
    plan = small_plan([4000, 5000])
    y = torch.zeros(plan.y_size, device="cuda")
    for kw in (dict(channel=2), dict(channel=-1), dict(hop=0), dict(n_mels=0), dict(n_mels=129),
               dict(f_lo=8000.0, f_hi=7000.0), dict(f_hi=8001.0), dict(log_floor=0.0), dict(stack=0),
               dict(stride=0), dict(fs=float("nan"))):
        with pytest.raises(RsimError):
            plan.log_mel(y, **kw)
