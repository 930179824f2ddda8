"""RIRs longer than one block of the largest FFT size reaches: uniformly
partitioned convolution (virtual sources delayed by whole parts, each with one
part of the RIRs) against the FP64 oracle's direct convolution with the whole
(cut) RIRs.  The planner sends an utterance there when its kept RIRs do not fit
one block -- always without a cut-off, and under a cut-off when the plan was made
with long_rirs -- and keeps the others on the regular path, so every batch here
mixes both.  Every gain mode and both output ranges; tolerances as for the
per-source path."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth
from parity_checks import close_vec, grads_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5
REACH = 3 * 16384 // 4 + 1          # taps one block of N = 16384 reaches


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def concat(*bs):
    """One batch holding the utterances of bs in order."""
    return synth.Batch(bs[0].num_mics,
                       np.concatenate([b.num_sources for b in bs]).astype(np.int32),
                       np.concatenate([b.num_samples for b in bs]).astype(np.int64),
                       np.concatenate([b.rir_len for b in bs]).astype(np.int32),
                       np.concatenate([b.x for b in bs]).astype(np.float32),
                       np.concatenate([b.rir for b in bs]).astype(np.float32),
                       np.concatenate([b.snr_db for b in bs]).astype(np.float32))


def no_cut_batch():
    """Untruncated RIRs of 7200-19200 taps (some beyond the reach, some within) and one
    utterance of short RIRs."""
    long = synth.trim_rirs(synth.make_batch(201, [1, 700, 20011, 33333], [1, 2, 3, 2], synth.linear_pair_array(),
                                            (0.9, 1.2)), 202, min_frac=0.5)
    short = synth.make_batch(204, [9000], [2], synth.linear_pair_array(), (0.2, 0.3))
    return concat(long, short)


def cut_batch():
    """At eta = 30 dB: two utterances whose kept RIRs exceed the reach (RT60 2.2-2.6 s,
    35-42 k taps untruncated) between two that fit."""
    mics = synth.linear_pair_array()
    long = synth.make_batch(301, [12000, 30011], [2, 3], mics, (2.2, 2.6))
    short = synth.make_batch(302, [900, 17000], [1, 2], mics, (0.3, 0.9))
    return concat(short.subset([0]), long.subset([0]), short.subset([1]), long.subset([1]))


def check_channels(y, ref, b, output_mode):
    n_out = synth.output_lengths(b, output_mode)
    off = 0
    for u in range(b.num_utts):
        n = int(n_out[u])
        for j in range(b.num_mics):
            close_vec(y[off:off + n], ref[off:off + n], f"y u={u} j={j}")
            off += n
    assert off == y.shape[0]


def run_and_check(b, eta, gain_mode, output_mode, long_rirs=False, fft_sizes=None, graphs=True, seed=0):
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=gain_mode, output_mode=output_mode, long_rirs=long_rirs,
                          fft_sizes=fft_sizes, graphs=graphs, snr_ref_mic=b.num_mics - 1)
    S, R = plan.S, plan.R
    x, rir = dev(b.x), dev(b.rir)
    rng = np.random.default_rng(seed)
    if gain_mode == 1:
        gains = dev(np.linspace(0.6, 1.3, S))
    elif gain_mode == 2:
        alpha_r = rng.uniform(-1.2, 1.2, R).astype(np.float32)
        gains = dev(alpha_r)
    else:
        gains = torch.empty(S, device="cuda")
    y = torch.full((plan.y_size,), float("nan"), device="cuda")
    tl = torch.empty(R, dtype=torch.int32, device="cuda")
    snr = dev(b.snr_db) if gain_mode in (0, 3) else None
    for _ in range(2):                       # with graphs the second call replays the captured graph
        plan.filter_mix(x, rir, gains, y, snr_db=snr, trunc_len=tl)
    plan.sync_status()
    L = oracle.truncate_batch(b, eta)["L"]
    np.testing.assert_array_equal(tl.cpu().numpy(), L)
    q = plan.query()
    ri = b.rir_index()
    np.testing.assert_array_equal(q["l_max"], [L[ri[u]:ri[u + 1]].max() for u in range(b.num_utts)])
    deferred = q["l_max"] > 3 * max(fft_sizes or [16384]) // 4 + 1
    assert np.all(q["log2_n"] > 0)
    # forward: from the oracle's own gains
    if gain_mode == 2:
        ref = oracle.forward_rir_gains(b, alpha_r.astype(np.float64), eta, output_mode=output_mode)
    else:
        if gain_mode == 0:
            alpha = oracle.forward(b, eta)["alpha"]
        elif gain_mode == 3:
            alpha, _ = oracle.reverberant_gains(b, eta_db=eta, ref_mic=b.num_mics - 1)
        else:
            alpha = gains.cpu().numpy().astype(np.float64)
        if gain_mode in (0, 3):
            np.testing.assert_allclose(gains.cpu().numpy(), alpha, rtol=REL, atol=0)
        ref = oracle.forward(b, eta, alpha=alpha, output_mode=output_mode)
    check_channels(y.cpu().numpy(), ref["y"], b, output_mode)
    # backward (the gains are inputs in every mode)
    gy = synth.grad_like(seed + 1, plan.y_size)
    gx, gr = torch.empty_like(x), torch.full_like(rir, float("nan"))
    gg = torch.empty(plan.G, device="cuda")
    plan.filter_mix_backward(dev(gy), x, gains, gx, gr, gg)
    plan.sync_status()
    a_in = gains.cpu().numpy().astype(np.float64)
    if gain_mode == 2:
        bw = oracle.backward_rir_gains(b, L, a_in, gy.astype(np.float64), output_mode=output_mode)
    else:
        bw = oracle.backward(b, L, a_in, gy.astype(np.float64), output_mode=output_mode)
    grads_close(b, bw, L, dx=gx.cpu().numpy(), dh=gr.cpu().numpy(), dalpha=gg.cpu().numpy())
    return plan, q, deferred


@pytest.mark.parametrize("gain_mode,output_mode,fft_sizes", [
    (1, 0, None), (0, 0, None), (1, 0, [8192]), (0, 0, [4096, 16384]),
    (1, 1, None), (2, 0, None), (2, 1, None), (3, 0, None), (3, 1, [8192]),
])
def test_partitioned_without_cut_off(gain_mode, output_mode, fft_sizes):
    b = no_cut_batch()
    assert b.rir_len.max() > 12289
    _, q, _ = run_and_check(b, math.inf, gain_mode, output_mode, fft_sizes=fft_sizes, seed=10 + gain_mode)
    # the short-RIR utterance stays on the regular path, the longest-RIR one does not
    n_max = 16384 if fft_sizes is None else max(fft_sizes)
    reach = 3 * n_max // 4 + 1
    assert q["l_max"][-1] <= reach and q["hop"][-1] == (1 << int(q["log2_n"][-1])) - q["l_max"][-1] + 1
    long_u = int(np.argmax(q["l_max"]))
    assert q["l_max"][long_u] > reach and q["hop"][long_u] == n_max // 2 + 1


@pytest.mark.parametrize("gain_mode,output_mode,graphs", [(0, 0, True), (1, 1, True), (2, 0, False), (2, 1, True),
                                                          (3, 1, True), (3, 0, False)])
def test_partitioned_under_a_cut_off(gain_mode, output_mode, graphs):
    b = cut_batch()
    L = oracle.truncate_batch(b, 30.0)["L"]
    ri = b.rir_index()
    lmax = np.array([L[ri[u]:ri[u + 1]].max() for u in range(b.num_utts)])
    assert np.all(lmax[[1, 3]] > REACH) and np.all(lmax[[0, 2]] <= REACH)
    _, q, deferred = run_and_check(b, 30.0, gain_mode, output_mode, long_rirs=True, graphs=graphs,
                                   seed=20 + gain_mode)
    np.testing.assert_array_equal(deferred, [False, True, False, True])
    np.testing.assert_array_equal(q["hop"][[1, 3]], 8193)          # blocks of the partitioned path


def test_kept_rir_beyond_the_reach_without_long_rirs_is_reported():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = cut_batch()
    plan = Plan.for_batch(b, eta_db=30.0, gain_mode=1)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(dev(b.x), dev(b.rir), dev(np.ones(plan.S)), y)
    with pytest.raises(RsimError) as e:
        plan.sync_status()
    assert e.value.status == 2


def test_small_largest_size_with_many_parts():
    # only N = 2048 allowed: parts of 1024 taps, 8 of them for one source
    b = synth.make_batch(43, [3000, 5000], [1, 2], synth.linear_pair_array(), (0.5, 0.5))
    assert oracle.truncate_batch(b, 60.0)["L"].max() > 3 * 2048 // 4 + 1
    run_and_check(b, 60.0, 1, 0, long_rirs=True, fft_sizes=[2048], seed=31)


def test_the_largest_number_of_virtual_sources():
    # 16 sources x 4 parts of 1024 taps (4000-tap RIRs, only N = 2048): the 64 virtual
    # sources a partitioned plan's utterance may hold
    b = synth.make_batch(47, [3000], [16], synth.linear_pair_array(), (0.25, 0.25))
    assert int(b.rir_len.max()) == 4000
    run_and_check(b, math.inf, 1, 0, fft_sizes=[2048], seed=33)


def test_too_many_parts_is_unsupported():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(212, [5000], [16], synth.linear_pair_array(), (2.5, 2.6))   # 16 x 5-6 parts > 64
    with pytest.raises(RsimError) as e:
        Plan.for_batch(b, eta_db=math.inf, gain_mode=1)
    assert e.value.status == 2


def test_partitioned_plan_cannot_be_reshaped():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = cut_batch()
    plan = Plan.for_batch(b, eta_db=30.0, gain_mode=1, long_rirs=True)
    with pytest.raises(RsimError) as e:
        plan.reshape_for(b.subset([0, 2]))
    assert e.value.status == 2
