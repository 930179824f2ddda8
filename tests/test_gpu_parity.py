"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Tolerances (fixed by the benchmark spec for this path): per output channel a
relative L2 error <= 1e-5 and a max-abs error <= 1e-5 x the channel's peak;
truncation lengths exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth
from parity_checks import grads_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def gpu_forward(batch, eta=20.0, fft_sizes=None, seg=0, gains=None, bseg=0):
    from paper_1712_03439_gb300 import Plan, filter_mix
    plan = Plan.for_batch(batch, eta_db=eta, fft_sizes=fft_sizes,
                          gain_mode=0 if gains is None else 1, segment_len=seg,
                          bwd_segment_len=bseg)
    x, rir = dev(batch.x), dev(batch.rir)
    if gains is None:
        out = filter_mix(plan, x, rir, snr_db=dev(batch.snr_db))
    else:
        out = filter_mix(plan, x, rir, gains=dev(gains))
    plan.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return plan, res, (x, rir, out["gains"])


def assert_channels_close(y, ref, batch, rel=REL_L2, mabs=MAX_ABS, what="y"):
    yo = batch.y_offsets()
    J = batch.num_mics
    for u in range(batch.num_utts):
        nx = int(batch.num_samples[u])
        for j in range(J):
            sl = slice(yo[u] + j * nx, yo[u] + (j + 1) * nx)
            g, r = y[sl].astype(np.float64), ref[sl]
            peak = np.abs(r).max()
            err = np.abs(g - r)
            if peak == 0:
                assert err.max() == 0, f"{what} u={u} j={j}: nonzero output for a zero reference"
                continue
            rl2 = np.linalg.norm(g - r) / np.linalg.norm(r)
            assert rl2 <= rel, f"{what} u={u} j={j}: rel L2 {rl2:.3e}"
            assert err.max() <= mabs * peak, f"{what} u={u} j={j}: max abs {err.max() / peak:.3e} x peak"


def small_batch(seed=7, lengths=(1, 700, 20011, 50000, 70001), n_src=(1, 2, 3, 4, 2),
                rt60=(0.1, 0.3), J=2):
    mics = synth.linear_pair_array() if J == 2 else synth.circular_array(J, 0.05)
    return synth.make_batch(seed, list(lengths), list(n_src), mics, rt60)


# ---------------------------------------------------------------------------
# truncation (Eq. 7-9): lengths exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("eta", [0.0, 10.0, 20.0, 30.0, math.inf])
def test_truncation_lengths_exact(eta):
    # without a cut-off the RIR itself must fit the largest FFT size (3N/4+1 taps)
    b = synth.config_home(n_utts=12) if math.isfinite(eta) else small_batch(rt60=(0.1, 0.5))
    _, res, _ = gpu_forward(b, eta=eta, seg=0)
    ref = oracle.truncate_batch(b, eta)
    np.testing.assert_array_equal(res["trunc_len"], ref["L"].astype(np.int32))
    frac = ref["e_kept"] / ref["e_tot"]
    np.testing.assert_allclose(res["energy_kept_frac"], frac, rtol=1e-5, atol=0)


def _hand_batch(rirs, nx=3000, eta=20.0):
    """One utterance per RIR, 1 source, 1 mic."""
    b = synth.make_batch(3, [nx] * len(rirs), [1] * len(rirs), np.zeros((1, 2)), (0.1, 0.1),
                         n_taps=8)
    b.rir = np.concatenate([np.asarray(r, np.float32) for r in rirs])
    b.rir_len = np.array([len(r) for r in rirs], np.int32)
    return b


def test_truncation_special_rirs():
    r = np.random.Generator(np.random.PCG64(4))
    dyadic = (2.0 ** -np.arange(60)) * r.choice([-1.0, 1.0], 60)
    rirs = [np.zeros(100), [0.3], [1.0, 0.5, -1.0, 0.25, 0.1, 0.0],
            [1.0, 0.01, 0.01, 0.5, 0.01, 0.01, 0.01, 0.01], dyadic, r.standard_normal(700)]
    for eta in [0.0, 10.0, 20.0, 47.0, math.inf]:
        b = _hand_batch(rirs)
        _, res, _ = gpu_forward(b, eta=eta, gains=np.ones(len(rirs), np.float32))
        ref = oracle.truncate_batch(b, eta)
        np.testing.assert_array_equal(res["trunc_len"], ref["L"].astype(np.int32), err_msg=f"eta={eta}")


# ---------------------------------------------------------------------------
# gains and forward
# ---------------------------------------------------------------------------
def test_gains_match_oracle():
    b = small_batch()
    _, res, _ = gpu_forward(b)
    ref = oracle.forward(b, 20.0)
    np.testing.assert_allclose(res["gains"], ref["alpha"], rtol=2e-6, atol=0)


def test_forward_parity_small_batch():
    b = small_batch()
    _, res, _ = gpu_forward(b, eta=20.0)
    ref = oracle.forward(b, 20.0)                 # the oracle's own gains from the SNRs
    np.testing.assert_allclose(res["gains"], ref["alpha"], rtol=2e-6, atol=0)
    assert_channels_close(res["y"], ref["y"], b)


@pytest.mark.parametrize("n", [2048, 4096, 8192, 16384])
def test_forward_parity_each_fft_size(n):
    # short RIRs (eta = 10 dB) so every size is admissible
    b = small_batch(seed=11, lengths=(3, 1500, 9000, 33333), n_src=(2, 1, 4, 3), rt60=(0.1, 0.2))
    tr = oracle.truncate_batch(b, 10.0)
    if tr["L"].max() > 3 * n // 4 + 1:
        pytest.skip("RIR too long for this size")
    g = np.linspace(0.5, 1.5, int(b.num_sources.sum())).astype(np.float32)
    plan, res, _ = gpu_forward(b, eta=10.0, fft_sizes=[n], gains=g)
    assert np.all(plan.query()["log2_n"] == int(math.log2(n)))
    ref = oracle.forward(b, 10.0, alpha=g.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)


def test_forward_no_truncation_multi_segment():
    b = small_batch(seed=12, lengths=(40000, 65000), n_src=(3, 2), rt60=(0.2, 0.25))
    g = np.array([1.0, 0.7, 0.2, 1.0, 0.4], np.float32)
    _, res, _ = gpu_forward(b, eta=math.inf, seg=16384, gains=g)
    ref = oracle.forward(b, math.inf, alpha=g.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)


def test_forward_edge_cases():
    # Nx = 1, single-tap RIRs, I = J = 1, a zero RIR, Nx shorter than the hop
    b = synth.make_batch(5, [1, 2, 17, 5000], [1, 2, 1, 3], np.zeros((1, 2)), (0.05, 0.1))
    ro = b.rir_offsets()
    rirs = [b.rir[ro[r]:ro[r + 1]].copy() for r in range(b.num_rirs)]
    rirs[0] = np.array([0.5], np.float32)
    rirs[1] = np.zeros(40, np.float32)
    b.rir = np.concatenate(rirs)
    b.rir_len = np.array([len(r) for r in rirs], np.int32)
    g = np.ones(int(b.num_sources.sum()), np.float32)
    _, res, _ = gpu_forward(b, eta=20.0, gains=g)
    ref = oracle.forward(b, 20.0, alpha=g.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)


def _long_tail_batch():
    # RIRs of 2.5k-2.9k taps kept whole (eta = inf) with N = 4096: the hop
    # (about 1.2k) is shorter than the tail, which then spans several blocks
    return small_batch(seed=15, lengths=(9000, 40000, 70001), n_src=(2, 3, 1), rt60=(0.16, 0.18))


def test_forward_tail_spanning_several_blocks():
    b = _long_tail_batch()
    g = np.linspace(0.4, 1.2, int(b.num_sources.sum())).astype(np.float32)
    plan, res, _ = gpu_forward(b, eta=math.inf, fft_sizes=[4096], seg=16384, gains=g)
    q = plan.query()
    assert np.all(q["l_max"] - 1 > q["hop"])           # the regime under test
    ref = oracle.forward(b, math.inf, alpha=g.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)


def test_backward_tail_spanning_several_blocks():
    b = _long_tail_batch()
    S = int(b.num_sources.sum())
    gains = np.linspace(0.4, 1.2, S).astype(np.float32)
    gy = synth.grad_like(23, b.y_size)
    _, gx, gr, gg = gpu_backward(b, math.inf, gains, gy, seg=16384, fft_sizes=[4096], bseg=16384)
    L = oracle.truncate_batch(b, math.inf)["L"]
    ref = oracle.backward(b, L, gains.astype(np.float64), gy)
    grads_close(b, ref, L, dx=gx, dh=gr, dalpha=gg)


def test_results_do_not_depend_on_segmentation():
    b = small_batch(seed=13, lengths=(90001, 140000, 31000), n_src=(2, 3, 1))
    ys = []
    for seg in [16384, 40000, 1 << 30]:
        _, res, _ = gpu_forward(b, eta=20.0, seg=seg)
        ys.append(res["y"])
    np.testing.assert_array_equal(ys[0], ys[1])
    np.testing.assert_array_equal(ys[0], ys[2])


def test_graph_replay_equals_eager_launch():
    from paper_1712_03439_gb300 import Plan
    b = small_batch(seed=16, lengths=(5000, 70000, 20000), n_src=(2, 1, 3))
    S = int(b.num_sources.sum())
    x, rir, snr = dev(b.x), dev(b.rir), dev(b.snr_db)
    gy = dev(synth.grad_like(24, b.y_size))
    outs = []
    for graphs in (False, True):
        plan = Plan.for_batch(b, eta_db=20.0, gain_mode=0, graphs=graphs)
        gains = torch.empty(S, device="cuda")
        y = torch.empty(b.y_size, device="cuda")
        gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty(S, device="cuda")
        for _ in range(3):                     # capture once, then replay
            y.fill_(7.0)
            gx.fill_(7.0)
            plan.filter_mix(x, rir, gains, y, snr_db=snr)
            plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
        plan.sync_status()
        outs.append([t.cpu().numpy() for t in (y, gains, gx, gr, gg)])
    for a, c in zip(*outs):
        np.testing.assert_array_equal(a, c)


def test_graph_replay_with_alternating_buffer_sets():
    # five pointer sets used round-robin (more than the plan keeps graphs for): every
    # replay or re-capture gives the eager result, and the sets do not leak into each other
    from paper_1712_03439_gb300 import Plan
    b = small_batch(seed=17, lengths=(9000, 30000), n_src=(3, 1))
    S = int(b.num_sources.sum())
    snr = dev(b.snr_db)
    ref_plan = Plan.for_batch(b, eta_db=20.0, gain_mode=0, graphs=False)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=0, graphs=True)
    sets = []
    for k in range(5):
        scale = 1.0 + 0.25 * k                    # different inputs per set
        x, rir = dev(b.x * scale), dev(b.rir)
        sets.append(dict(x=x, rir=rir, gy=dev(synth.grad_like(30 + k, b.y_size)),
                         gains=torch.empty(S, device="cuda"), y=torch.empty(b.y_size, device="cuda"),
                         gx=torch.empty_like(x), gr=torch.empty_like(rir), gg=torch.empty(S, device="cuda")))
    for rnd in range(3):
        for k, T in enumerate(sets):
            T["y"].fill_(7.0)
            plan.filter_mix(T["x"], T["rir"], T["gains"], T["y"], snr_db=snr)
            plan.filter_mix_backward(T["gy"], T["x"], T["gains"], T["gx"], T["gr"], T["gg"])
            if rnd == 2:
                R = {n: torch.empty_like(v) for n, v in T.items() if n in ("gains", "y", "gx", "gr", "gg")}
                ref_plan.filter_mix(T["x"], T["rir"], R["gains"], R["y"], snr_db=snr)
                ref_plan.filter_mix_backward(T["gy"], T["x"], R["gains"], R["gx"], R["gr"], R["gg"])
                for n in R:
                    np.testing.assert_array_equal(T[n].cpu().numpy(), R[n].cpu().numpy())
    plan.sync_status()


def _merge(a, b):
    return synth.Batch(a.num_mics, np.concatenate([a.num_sources, b.num_sources]),
                       np.concatenate([a.num_samples, b.num_samples]),
                       np.concatenate([a.rir_len, b.rir_len]), np.concatenate([a.x, b.x]),
                       np.concatenate([a.rir, b.rir]), np.concatenate([a.snr_db, b.snr_db]))


@pytest.mark.parametrize("n_fft", [2048, 8192])
def test_longest_admissible_rir_and_one_tap_more(n_fft):
    # L_max = 3N/4 + 1 is the longest kept RIR a size admits (hop = N/4, the carry spans
    # three blocks): exact against the oracle; one tap more (no cut-off) goes through the
    # partitioned convolution, exact as well
    lmax = 3 * n_fft // 4 + 1
    rng = np.random.Generator(np.random.PCG64(n_fft))

    def batch(nh):
        b = small_batch(seed=80 + nh % 7, lengths=(3 * n_fft + 77, 5000), n_src=(2, 1))
        lens = [nh, nh - 5, nh // 2, 17, nh, 3]            # (u0: i0 j0, i0 j1, i1 j0, i1 j1), (u1: ...)
        rirs = [rng.normal(0, 0.1, L).astype(np.float32) for L in lens]
        for h in rirs:
            h[-1] = 0.05                                    # nonzero last tap: L = Nh without cut-off
        return synth.Batch(b.num_mics, b.num_sources, b.num_samples, np.array(lens, np.int32),
                           b.x, np.concatenate(rirs), b.snr_db)

    b = batch(lmax)
    gains = np.array([1.0, 0.7, 1.2], np.float32)
    plan, res, _ = gpu_forward(b, eta=math.inf, fft_sizes=[n_fft], gains=gains)
    assert plan.query()["hop"][0] == n_fft // 4
    ref = oracle.forward(b, math.inf, alpha=gains.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)
    b1 = batch(lmax + 1)
    _, res1, _ = gpu_forward(b1, eta=math.inf, fft_sizes=[n_fft], gains=gains)
    assert_channels_close(res1["y"], oracle.forward(b1, math.inf, alpha=gains.astype(np.float64))["y"], b1)


def test_minority_fft_size_moves_to_the_dominant_one():
    # two short utterances with short RIRs would pick a small N on their own; beside
    # thirty long ones they take the batch's dominant size, and the results stay exact
    from paper_1712_03439_gb300 import Plan
    big = synth.make_batch(61, [96000] * 30, [2] * 30, synth.linear_pair_array(), (0.3, 0.35))
    small = synth.make_batch(62, [2500, 3100], [1, 2], synth.linear_pair_array(), (0.02, 0.03))
    b = _merge(big, small)
    S = int(b.num_sources.sum())
    gains = np.linspace(0.8, 1.2, S).astype(np.float32)
    plan, res, _ = gpu_forward(b, eta=20.0, gains=gains)
    n = plan.query()["log2_n"]
    assert len(set(n.tolist())) == 1, n
    alone, _, _ = gpu_forward(small, eta=20.0, gains=gains[-3:])
    assert alone.query()["log2_n"].max() < n[0]       # on their own they choose smaller sizes
    sub = b.subset([30, 31])
    ref = oracle.forward(sub, 20.0, alpha=gains[-3:].astype(np.float64))
    yo = b.y_offsets()
    assert_channels_close(res["y"][yo[30]:yo[32]], ref["y"], sub)


def test_results_do_not_depend_on_utterance_order():
    b = small_batch(seed=14, lengths=(5000, 70000, 20000, 45000), n_src=(2, 1, 4, 3))
    perm = [2, 0, 3, 1]
    bp = b.subset(perm)
    _, r0, _ = gpu_forward(b)
    _, r1, _ = gpu_forward(bp)
    yo, yp = b.y_offsets(), bp.y_offsets()
    for k, u in enumerate(perm):
        np.testing.assert_array_equal(r0["y"][yo[u]:yo[u + 1]], r1["y"][yp[k]:yp[k + 1]])


def test_full_size_home_workload_sampled_utterances():
    # the 256-utterance Google-Home-like batch at full size, in the benchmark's
    # launch configuration; the oracle checks a sample of its utterances
    b = synth.config_home()
    _, res, _ = gpu_forward(b, eta=20.0)
    rng = np.random.Generator(np.random.PCG64(1))
    pick = sorted(rng.choice(b.num_utts, 3, replace=False).tolist())
    sub = b.subset(pick)
    si = b.src_index()
    ref = oracle.forward(sub, 20.0)               # the oracle's own gains from the SNRs
    got_alpha = np.concatenate([res["gains"][si[u]:si[u + 1]] for u in pick])
    np.testing.assert_allclose(got_alpha, ref["alpha"], rtol=2e-6, atol=0)
    yo = b.y_offsets()
    y = np.concatenate([res["y"][yo[u]:yo[u + 1]] for u in pick])
    assert_channels_close(y, ref["y"], sub)
    tr = oracle.truncate_batch(b, 20.0)
    np.testing.assert_array_equal(res["trunc_len"], tr["L"].astype(np.int32))


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------
def gpu_backward(batch, eta, gains, gy, seg=0, fft_sizes=None, bseg=0):
    from paper_1712_03439_gb300 import Plan
    plan, res, (x, rir, g) = gpu_forward(batch, eta=eta, gains=gains, seg=seg, fft_sizes=fft_sizes,
                                         bseg=bseg)
    gx = torch.empty_like(x)
    gr = torch.empty_like(rir)
    gg = torch.empty_like(g)
    plan.filter_mix_backward(dev(gy), x, g, gx, gr, gg)
    plan.sync_status()
    return res, gx.cpu().numpy(), gr.cpu().numpy(), gg.cpu().numpy()


@pytest.mark.parametrize("eta,seg,bseg", [(20.0, 0, 0), (math.inf, 16384, 16384), (20.0, 0, 40000)])
def test_backward_parity_small_batch(eta, seg, bseg):
    b = small_batch(seed=21, lengths=(900, 20011, 50000, 70001), n_src=(2, 3, 4, 1))
    S = int(b.num_sources.sum())
    gains = np.linspace(0.6, 1.3, S).astype(np.float32)
    gy = synth.grad_like(22, b.y_size)
    _, gx, gr, gg = gpu_backward(b, eta, gains, gy, seg=seg, bseg=bseg)
    L = oracle.truncate_batch(b, eta)["L"]
    ref = oracle.backward(b, L, gains.astype(np.float64), gy)
    # per source: dx; per RIR: dh; dalpha elementwise
    grads_close(b, ref, L, dx=gx, dh=gr, dalpha=gg)


def test_autograd_function_matches_oracle_gradient():
    from paper_1712_03439_gb300 import Plan, filter_mix_autograd
    b = synth.config_fd_subcase()
    S = int(b.num_sources.sum())
    gains = np.linspace(0.6, 1.4, S).astype(np.float32)
    t = synth.grad_like(6, b.y_size)
    plan = Plan.for_batch(b, eta_db=math.inf, gain_mode=1)
    x = dev(b.x).requires_grad_(True)
    rir = dev(b.rir).requires_grad_(True)
    g = dev(gains).requires_grad_(True)
    y = filter_mix_autograd(plan, x, rir, g)
    loss = 0.5 * torch.sum((y - dev(t)) ** 2)
    loss.backward()
    L = oracle.truncate_batch(b, math.inf)["L"]
    yref = oracle.forward(b, math.inf, alpha=gains.astype(np.float64))["y"]
    ref = oracle.backward(b, L, gains.astype(np.float64), yref - t)
    grads_close(b, ref, L, dx=x.grad.cpu().numpy(), dh=rir.grad.cpu().numpy(), dalpha=g.grad.cpu().numpy())


def test_backward_each_fft_size():
    b = small_batch(seed=31, lengths=(7000, 23000), n_src=(2, 3), rt60=(0.1, 0.15))
    S = int(b.num_sources.sum())
    gains = np.linspace(0.5, 1.2, S).astype(np.float32)
    gy = synth.grad_like(32, b.y_size)
    L = oracle.truncate_batch(b, 10.0)["L"]
    ref = oracle.backward(b, L, gains.astype(np.float64), gy)
    for n in [2048, 4096, 8192, 16384]:
        if L.max() > 3 * n // 4 + 1:
            continue
        _, gx, gr, gg = gpu_backward(b, 10.0, gains, gy, fft_sizes=[n])
        grads_close(b, ref, L, dx=gx, dh=gr, dalpha=gg, what=f"N={n} ")


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_backward_before_forward_is_a_state_error():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = small_batch(seed=41, lengths=(1000,), n_src=(1,))
    plan = Plan.for_batch(b, gain_mode=1)
    z = lambda n: torch.zeros(n, device="cuda")
    with pytest.raises(RsimError) as e:
        plan.filter_mix_backward(z(plan.y_size), z(plan.x_size), z(plan.S), z(plan.x_size),
                                 z(plan.rir_size), z(plan.S))
    assert e.value.status == 6


def test_silent_noise_source_is_reported():
    from paper_1712_03439_gb300._lib import RsimError
    b = small_batch(seed=42, lengths=(3000,), n_src=(2,))
    xo = b.x_offsets()
    b.x[xo[1]:xo[2]] = 0
    with pytest.raises(RsimError) as e:
        gpu_forward(b)
    assert e.value.status == 1


def test_rir_too_long_for_allowed_sizes_is_reported():
    # with a cut-off the kept lengths are known on the device only: a kept RIR beyond
    # 3N/4 + 1 taps for every allowed N is reported (without a cut-off such RIRs go
    # through the partitioned convolution)
    from paper_1712_03439_gb300._lib import RsimError
    b = small_batch(seed=43, lengths=(3000,), n_src=(1,), rt60=(0.5, 0.5))
    assert oracle.truncate_batch(b, 60.0)["L"].max() > 3 * 2048 // 4 + 1
    with pytest.raises(RsimError) as e:
        gpu_forward(b, eta=60.0, fft_sizes=[2048], gains=np.ones(1, np.float32))
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# microphone groups: J > 2 (8-mic circle as in the long-reverberation
# workload, shortened) and an odd J
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("J", [3, 8])
def test_forward_and_backward_many_mics(J):
    b = small_batch(seed=40 + J, lengths=(20000, 47000), n_src=(4, 2), rt60=(0.1, 0.25), J=J)
    S = int(b.num_sources.sum())
    gains = np.linspace(0.5, 1.3, S).astype(np.float32)
    gy = synth.grad_like(41, b.y_size)
    res, gx, gr, gg = gpu_backward(b, 20.0, gains, gy, seg=16384, bseg=16384)
    L = oracle.truncate_batch(b, 20.0)["L"]
    ref = oracle.forward(b, 20.0, alpha=gains.astype(np.float64))
    assert_channels_close(res["y"], ref["y"], b)
    gref = oracle.backward(b, L, gains.astype(np.float64), gy)
    grads_close(b, gref, L, dx=gx, dh=gr, dalpha=gg)
