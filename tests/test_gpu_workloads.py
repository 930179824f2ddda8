"""The stated workloads as parity cases (CUDA path vs the FP64 oracle).

* tiny: 1 s, 1 source, 1 mic, one 4800-tap RIR, N = 8192 -- compared in full;
* differentiable mix: the Google-Home recipe at 64 utterances through the
  autograd function with an L2 loss; the oracle checks sampled utterances;
* long reverberant multi-mic: 30 s utterances, 4 sources, 8 mics, RT60
  0.8-1.2 s, cut-offs of 10, 20 and 30 dB and none (two utterances of that shape);
  lengths exact, outputs, dx and dh (sampled RIRs) on sampled windows
  against the oracle's window forms, and the adjoint identities over the
  whole batch;
  without a cut-off (RIRs up to 19200 taps, beyond what one block of the
  largest FFT size reaches) through the partitioned convolution; and the same
  shape at 30 dB with the full output, one utterance whose kept RIRs fit a block
  beside one (RT60 2.0-2.4 s) whose kept RIRs do not.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth

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


def close_channel(g, r, what):
    g = g.astype(np.float64)
    peak = np.abs(r).max()
    if peak == 0:
        assert np.abs(g).max() == 0, what
        return
    rl2 = np.linalg.norm(g - r) / np.linalg.norm(r)
    assert rl2 <= REL_L2, f"{what}: rel L2 {rl2:.3e}"
    assert np.abs(g - r).max() <= MAX_ABS * peak, f"{what}: max abs {np.abs(g - r).max() / peak:.3e} x peak"


# ---------------------------------------------------------------------------
def test_tiny_workload_in_full():
    from paper_1712_03439_gb300 import Plan, filter_mix
    b = synth.config_tiny()
    assert b.num_samples[0] == 16000 and b.rir_len[0] == 4800
    plan = Plan.for_batch(b, eta_db=20.0, fft_sizes=[8192])
    out = filter_mix(plan, dev(b.x), dev(b.rir), snr_db=dev(b.snr_db))
    plan.sync_status()
    assert plan.query()["log2_n"][0] == 13
    ref = oracle.forward(b, 20.0)
    np.testing.assert_array_equal(out["trunc_len"].cpu().numpy(), ref["L"].astype(np.int32))
    close_channel(out["y"].cpu().numpy(), ref["y"], "tiny y")


# ---------------------------------------------------------------------------
def test_differentiable_mix_64_utterances_autograd():
    from paper_1712_03439_gb300 import Plan, filter_mix_autograd
    b = synth.config_diff()
    assert b.num_utts == 64
    S = int(b.num_sources.sum())
    gains = np.linspace(0.6, 1.4, S).astype(np.float32)
    t = synth.grad_like(61, b.y_size)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1)
    x = dev(b.x).requires_grad_(True)
    rir = dev(b.rir).requires_grad_(True)
    g = dev(gains).requires_grad_(True)
    y = filter_mix_autograd(plan, x, rir, g)
    loss = 0.5 * torch.sum((y - dev(t)) ** 2)
    loss.backward()
    yg = y.detach().cpu().numpy()
    resid = (y.detach() - dev(t)).cpu().numpy()          # the upstream gradient autograd passed
    L = oracle.truncate_batch(b, 20.0)["L"]
    pick = [3, 29, 60]
    sub = b.subset(pick)
    si, yo, xo, ri, ro = b.src_index(), b.y_offsets(), b.x_offsets(), b.rir_index(), b.rir_offsets()
    a_sub = np.concatenate([gains[si[u]:si[u + 1]] for u in pick]).astype(np.float64)
    L_sub = np.concatenate([L[ri[u]:ri[u + 1]] for u in pick])
    g_sub = np.concatenate([resid[yo[u]:yo[u + 1]] for u in pick])
    yref = oracle.forward(sub, 20.0, alpha=a_sub)["y"]
    gref = oracle.backward(sub, L_sub, a_sub, g_sub)
    so, sro, syo = sub.x_offsets(), sub.rir_offsets(), sub.y_offsets()
    gx, gr, gg = x.grad.cpu().numpy(), rir.grad.cpu().numpy(), g.grad.cpu().numpy()
    for k, u in enumerate(pick):
        J, nx = b.num_mics, int(b.num_samples[u])
        for j in range(J):
            close_channel(yg[yo[u] + j * nx:yo[u] + (j + 1) * nx],
                          yref[syo[k] + j * nx:syo[k] + (j + 1) * nx], f"y u={u} j={j}")
        for i in range(int(b.num_sources[u])):
            s, ss = si[u] + i, sub.src_index()[k] + i
            close_channel(gx[xo[s]:xo[s + 1]], gref["dx"][so[ss]:so[ss + 1]], f"dx u={u} i={i}")
        for q in range(ri[u + 1] - ri[u]):
            r, rs = ri[u] + q, sub.rir_index()[k] + q
            close_channel(gr[ro[r]:ro[r + 1]], gref["dh"][sro[rs]:sro[rs + 1]], f"dh u={u} r={q}")
        s0 = si[u]
        np.testing.assert_allclose(gg[s0:si[u + 1]], gref["dalpha"][sub.src_index()[k]:sub.src_index()[k + 1]],
                                   rtol=REL_L2, atol=REL_L2 * np.abs(gref["dalpha"]).max())


# ---------------------------------------------------------------------------
SEED_LONG = 171203439 + 40


@pytest.fixture(scope="module")
def long_batch():
    return synth.config_long(n_utts=2)


def check_long(b, eta, output_mode=0, long_rirs=False):
    """Forward + backward of a long-reverberation batch: lengths exact, adjoint
    identities over the whole batch, outputs, dx and dh on sampled windows against
    the oracle's window forms.  Returns the plan's query."""
    from paper_1712_03439_gb300 import Plan
    J, S = b.num_mics, int(b.num_sources.sum())
    gains = np.linspace(0.7, 1.3, S).astype(np.float32)
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=1, output_mode=output_mode, long_rirs=long_rirs)
    x, rir, g = dev(b.x), dev(b.rir), dev(gains)
    y = torch.empty(plan.y_size, device="cuda")
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    plan.filter_mix(x, rir, g, y, trunc_len=tl)
    gy = synth.grad_like(71, plan.y_size)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
    plan.filter_mix_backward(dev(gy), x, g, gx, gr, gg)
    plan.sync_status()
    q = plan.query()
    L = oracle.truncate_batch(b, eta)["L"]
    np.testing.assert_array_equal(tl.cpu().numpy(), L.astype(np.int32))
    yv, gxv, grv, ggv = (t.cpu().numpy() for t in (y, gx, gr, gg))
    # adjoint identities over the whole batch (FP64 sums of the GPU outputs)
    hhat = b.rir.astype(np.float64).copy()
    ro = b.rir_offsets()
    for r in range(b.num_rirs):
        hhat[ro[r] + L[r]:ro[r + 1]] = 0.0
    lhs = float(np.dot(gy.astype(np.float64), yv))
    for what, val in (("dx", np.dot(gxv.astype(np.float64), b.x.astype(np.float64))),
                      ("dh", np.dot(grv.astype(np.float64), hhat)),
                      ("dalpha", np.dot(ggv.astype(np.float64), gains.astype(np.float64)))):
        assert abs(val - lhs) <= REL_L2 * abs(lhs), f"<{what}, .> vs <g, y>: {abs(val - lhs) / abs(lhs):.3e}"
    # sampled windows: the oracle computes those output (and dx) positions only
    n_out = synth.output_lengths(b, output_mode)
    yo = np.concatenate([[0], np.cumsum(n_out * J)]).astype(np.int64)
    si, xo, ri = b.src_index(), b.x_offsets(), b.rir_index()
    W = 1000
    for u in range(b.num_utts):
        nx, ny = int(b.num_samples[u]), int(n_out[u])
        I = int(b.num_sources[u])
        xs = np.stack([b.x[xo[s]:xo[s + 1]] for s in range(si[u], si[u + 1])])
        rirs = [b.rir[ro[r]:ro[r + 1]] for r in range(ri[u], ri[u + 1])]
        Lu = L[ri[u]:ri[u + 1]]
        a_u = gains[si[u]:si[u + 1]].astype(np.float64)
        gu = gy[yo[u]:yo[u + 1]].reshape(J, ny)
        # (a window across the end of x only where the output runs past it)
        for n0 in sorted({0, 123457, ny - W} | ({nx - W // 2} if ny > nx else set())):
            yw = oracle.mix_window(xs, rirs, Lu, a_u, n0, n0 + W)
            for j in range(J):
                close_channel(yv[yo[u] + j * ny + n0:yo[u] + j * ny + n0 + W], yw[j], f"y u={u} j={j} n0={n0}")
        for m0 in (0, 250001, nx - W):
            for i in range(I):
                s = si[u] + i
                dxw = oracle.dx_window(gu, rirs, Lu, i, a_u[i], m0, m0 + W)
                close_channel(gxv[xo[s] + m0:xo[s] + m0 + W], dxw, f"dx u={u} i={i} m0={m0}")
        # dh of sampled RIRs element by element on tap windows: the start, the middle,
        # the window across the cut-off (zero from L on) and the last taps
        WH = 256
        for q_ in sorted({0, 5, 13, I * J - 1}):
            r, i, j = ri[u] + q_, q_ // J, q_ % J
            nh, Lr = int(b.rir_len[r]), int(L[r])
            for k0 in sorted({0, Lr // 2, max(Lr - WH // 2, 0), max(nh - WH, 0)}):
                k1 = min(k0 + WH, nh)
                dhw = oracle.dh_window(xs[i], gu[j], Lr, a_u[i], k0, k1)
                close_channel(grv[ro[r] + k0:ro[r] + k1], dhw, f"dh u={u} r={q_} k0={k0}")
    return q


@pytest.mark.parametrize("eta", [10.0, 20.0, 30.0, math.inf])
def test_long_reverberant_multimic(long_batch, eta):
    b = long_batch
    assert b.num_mics == 8 and np.all(b.num_sources == 4) and np.all(b.num_samples == 30 * synth.FS)
    check_long(b, eta)


def test_long_reverberant_full_output_with_kept_rirs_beyond_one_block():
    # the long-reverberation shape (30 s, 4 sources, 8-mic circle) at 30 dB: an utterance
    # at RT60 1.2-1.4 s whose kept RIRs fit one block of N = 16384 beside one at 2.0-2.4 s
    # whose kept RIRs do not (its partitioned path: up to 5 parts of 8192 taps), full output
    mics = synth.circular_array(8, 0.05)
    a = synth.make_batch(SEED_LONG, [30 * synth.FS], [4], mics, (1.2, 1.4))
    c = synth.make_batch(SEED_LONG + 1, [30 * synth.FS], [4], mics, (2.0, 2.4))
    b = synth.Batch(8, np.concatenate([a.num_sources, c.num_sources]), np.concatenate([a.num_samples, c.num_samples]),
                    np.concatenate([a.rir_len, c.rir_len]), np.concatenate([a.x, c.x]),
                    np.concatenate([a.rir, c.rir]), np.concatenate([a.snr_db, c.snr_db]))
    L = oracle.truncate_batch(b, 30.0)["L"]
    reach = 3 * 16384 // 4 + 1
    assert L[:32].max() <= reach < L[32:].max()
    q = check_long(b, 30.0, output_mode=1, long_rirs=True)
    np.testing.assert_array_equal(q["hop"], [(1 << int(q["log2_n"][0])) - q["l_max"][0] + 1, 8193])
