"""Per-(source, microphone) gains (gain mode 2, Eq. 2's alpha_ij): CUDA path
vs the FP64 oracle through the C-ABI, with the tolerances of the per-source
path (per channel or per vector a relative L2 error <= 1e-5, max-abs <= 1e-5
x peak; gain gradients elementwise within 1e-5 of the largest)."""
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


def close(a, r, what):
    close_vec(a, r, what)


def channels_close(y, ref, b):
    yo = b.y_offsets()
    for u in range(b.num_utts):
        n = int(b.num_samples[u])
        for j in range(b.num_mics):
            s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
            r = ref[s]
            if not np.any(r):
                assert not np.any(y[s]), f"u={u} j={j}"
                continue
            g = y[s].astype(np.float64)
            assert np.linalg.norm(g - r) <= REL * np.linalg.norm(r), f"y u={u} j={j}"
            assert np.max(np.abs(g - r)) <= REL * np.max(np.abs(r)), f"y u={u} j={j} max abs"


def run(b, alpha_r, gy, eta):
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=2, segment_len=16384, bwd_segment_len=16384)
    x, rir, a = dev(b.x), dev(b.rir), dev(alpha_r)
    y = torch.empty(plan.y_size, device="cuda")
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    plan.filter_mix(x, rir, a, y, trunc_len=tl)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty(plan.R, device="cuda")
    plan.filter_mix_backward(dev(gy), x, a, gx, gr, gg)
    plan.sync_status()
    return dict(y=y.cpu().numpy(), L=tl.cpu().numpy(), dx=gx.cpu().numpy(), dh=gr.cpu().numpy(),
                da=gg.cpu().numpy())


@pytest.mark.parametrize("J,eta", [(2, 20.0), (3, math.inf), (8, 20.0)])
def test_rir_gains_match_oracle(J, eta):
    mics = synth.linear_pair_array() if J == 2 else synth.circular_array(J, 0.05)
    b = synth.trim_rirs(synth.make_batch(61 + J, [900, 20011, 50000, 33333], [2, 3, 1, 4], mics, (0.1, 0.25)),
                        62 + J)
    rng = np.random.default_rng(J)
    alpha_r = rng.uniform(-1.2, 1.2, b.num_rirs).astype(np.float32)
    gy = synth.grad_like(63 + J, b.y_size)
    got = run(b, alpha_r, gy, eta)
    ref = oracle.forward_rir_gains(b, alpha_r.astype(np.float64), eta)
    np.testing.assert_array_equal(got["L"], ref["L"])
    channels_close(got["y"], ref["y"], b)
    bw = oracle.backward_rir_gains(b, ref["L"], alpha_r.astype(np.float64), gy.astype(np.float64))
    grads_close(b, bw, ref["L"], dx=got["dx"], dh=got["dh"], dalpha=got["da"])


def test_per_source_gains_given_per_rir_reproduce_mode_1():
    from paper_1712_03439_gb300 import Plan
    b = synth.make_batch(71, [5000, 30000], [3, 2], synth.linear_pair_array(), (0.1, 0.2))
    S = int(b.num_sources.sum())
    alpha_s = np.linspace(0.4, 1.3, S).astype(np.float32)
    gy = synth.grad_like(72, b.y_size)
    two = run(b, np.repeat(alpha_s, b.num_mics), gy, 20.0)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, segment_len=16384, bwd_segment_len=16384)
    x, rir, a = dev(b.x), dev(b.rir), dev(alpha_s)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(x, rir, a, y)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty(S, device="cuda")
    plan.filter_mix_backward(dev(gy), x, a, gx, gr, gg)
    plan.sync_status()
    close(two["y"], y.cpu().numpy().astype(np.float64), "y")
    close(two["dx"], gx.cpu().numpy().astype(np.float64), "dx")
    close(two["dh"], gr.cpu().numpy().astype(np.float64), "dh")
    np.testing.assert_allclose(two["da"].reshape(S, b.num_mics).sum(1), gg.cpu().numpy(), rtol=1e-4,
                               atol=1e-5 * np.abs(gg.cpu().numpy()).max())


def test_gain_gradient_follows_the_last_forwards_rirs():
    """The gain gradient reads the RIRs of the last forward; a forward with another
    RIR buffer (replayed graphs included) must not leave a stale pointer behind."""
    from paper_1712_03439_gb300 import Plan
    b = synth.make_batch(81, [8000, 12000], [2, 1], synth.linear_pair_array(), (0.1, 0.2))
    alpha_r = np.linspace(0.5, 1.5, b.num_rirs).astype(np.float32)
    gy = synth.grad_like(82, b.y_size)
    plan = Plan.for_batch(b, eta_db=math.inf, gain_mode=2)
    x, a, g = dev(b.x), dev(alpha_r), dev(gy)
    y = torch.empty(plan.y_size, device="cuda")
    gx, gg = torch.empty_like(x), torch.empty(plan.R, device="cuda")
    rirs = [dev(b.rir), dev(0.5 * b.rir)]
    results = []
    for k in (0, 1, 0, 1):
        gr = torch.empty_like(rirs[k])
        plan.filter_mix(x, rirs[k], a, y)
        plan.filter_mix_backward(g, x, a, gx, gr, gg)
        plan.sync_status()
        results.append(gg.cpu().numpy().copy())
    np.testing.assert_allclose(results[1], 0.5 * results[0], rtol=1e-5, atol=1e-7)
    np.testing.assert_array_equal(results[2], results[0])
    np.testing.assert_array_equal(results[3], results[1])


def test_autograd_with_rir_gains():
    from paper_1712_03439_gb300 import Plan, filter_mix_autograd
    b = synth.config_fd_subcase()
    alpha_r = np.linspace(-0.8, 1.2, b.num_rirs).astype(np.float32)
    t = synth.grad_like(91, b.y_size)
    plan = Plan.for_batch(b, eta_db=math.inf, gain_mode=2)
    x = dev(b.x).requires_grad_(True)
    rir = dev(b.rir).requires_grad_(True)
    g = dev(alpha_r).requires_grad_(True)
    y = filter_mix_autograd(plan, x, rir, g)
    (0.5 * torch.sum((y - dev(t)) ** 2)).backward()
    ref = oracle.forward_rir_gains(b, alpha_r.astype(np.float64), math.inf)
    bw = oracle.backward_rir_gains(b, ref["L"], alpha_r.astype(np.float64), ref["y"] - t)
    grads_close(b, bw, ref["L"], dx=x.grad.cpu().numpy(), dh=rir.grad.cpu().numpy(), dalpha=g.grad.cpu().numpy())


def test_autograd_with_rir_gains_and_a_non_contiguous_rir():
    # the forward makes a contiguous copy of rir; the gain gradient reads that copy
    # in the backward, so it must outlive the forward call
    from paper_1712_03439_gb300 import Plan, filter_mix_autograd
    b = synth.config_fd_subcase()
    alpha_r = np.linspace(-0.8, 1.2, b.num_rirs).astype(np.float32)
    t = synth.grad_like(92, b.y_size)
    plan = Plan.for_batch(b, eta_db=math.inf, gain_mode=2)
    x = dev(b.x).requires_grad_(True)
    wide = torch.zeros((b.rir.shape[0], 2), device="cuda")
    wide[:, 0] = dev(b.rir)
    wide.requires_grad_(True)
    rir = wide[:, 0]                              # stride 2: not contiguous
    assert not rir.is_contiguous()
    g = dev(alpha_r).requires_grad_(True)
    y = filter_mix_autograd(plan, x, rir, g)
    junk = [torch.full((b.rir.shape[0],), 9.0, device="cuda") for _ in range(4)]   # reuse freed blocks
    (0.5 * torch.sum((y - dev(t)) ** 2)).backward()
    del junk
    ref = oracle.forward_rir_gains(b, alpha_r.astype(np.float64), math.inf)
    bw = oracle.backward_rir_gains(b, ref["L"], alpha_r.astype(np.float64), ref["y"] - t)
    grads_close(b, bw, ref["L"], dx=x.grad.cpu().numpy(), dh=wide.grad[:, 0].cpu().numpy(),
                dalpha=g.grad.cpu().numpy())


@pytest.mark.parametrize("gain_mode", [1, 2])
def test_autograd_two_forwards_then_two_backwards(gain_mode):
    # gradient accumulation on one plan: both forwards run before either backward;
    # each backward must see its own forward's RIRs, cut-off and spectra
    from paper_1712_03439_gb300 import Plan, filter_mix_autograd
    b = synth.make_batch(93, [6000, 15000], [2, 3], synth.linear_pair_array(), (0.1, 0.3))
    G = b.num_rirs if gain_mode == 2 else int(b.num_sources.sum())
    alpha = np.linspace(0.5, 1.4, G).astype(np.float32)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=gain_mode)
    t = synth.grad_like(94, b.y_size)
    grads = []
    for scale in (1.0, 0.5):
        x = dev(b.x).requires_grad_(True)
        rir = dev(scale * b.rir).requires_grad_(True)
        g = dev(alpha).requires_grad_(True)
        grads.append((x, rir, g))
    ys = [filter_mix_autograd(plan, *v) for v in grads]
    for y in ys:
        (0.5 * torch.sum((y - dev(t)) ** 2)).backward()
    for (x, rir, g), scale in zip(grads, (1.0, 0.5)):
        bs = synth.Batch(b.num_mics, b.num_sources, b.num_samples, b.rir_len, b.x,
                         (scale * b.rir).astype(np.float32), b.snr_db)
        L = oracle.truncate_batch(bs, 20.0)["L"]
        if gain_mode == 2:
            ref = oracle.forward_rir_gains(bs, alpha.astype(np.float64), 20.0)
            bw = oracle.backward_rir_gains(bs, ref["L"], alpha.astype(np.float64), ref["y"] - t)
        else:
            ref = oracle.forward(bs, 20.0, alpha=alpha.astype(np.float64))
            bw = oracle.backward(bs, L, alpha.astype(np.float64), ref["y"] - t)
        grads_close(bs, bw, L, dx=x.grad.cpu().numpy(), dh=rir.grad.cpu().numpy(), dalpha=g.grad.cpu().numpy(),
                    what=f"scale {scale} ")
