"""Full-length output (output_mode 1): CUDA path vs the FP64 oracle.

Ny = Nx + (longest RIR of the utterance) - 1 samples per microphone; the
output is the full convolution of Eq. 2, exactly zero from Nx + L_max - 1 on.
Same tolerances as the "same"-output parity tests: per channel a relative L2
error <= 1e-5 and a max-abs error <= 1e-5 x the channel's peak.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03439_gb300 import synth
from parity_checks import close_vec, grads_close

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float32)


def full_batch(seed=31):
    b = synth.make_batch(seed, [1, 700, 20011, 50000, 33333], [1, 2, 3, 2, 4],
                         synth.linear_pair_array(), (0.1, 0.3))
    return synth.trim_rirs(b, seed + 1)


def run(batch, eta, gains, gy=None, seg=0, bseg=0, fft_sizes=None):
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(batch, eta_db=eta, gain_mode=1, segment_len=seg, bwd_segment_len=bseg,
                          fft_sizes=fft_sizes, output_mode=1)
    x, rir, g = dev(batch.x), dev(batch.rir), dev(gains)
    y = torch.full((plan.y_size,), float("nan"), device="cuda")   # every sample must be written
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    plan.filter_mix(x, rir, g, y, trunc_len=tl)
    out = {"y": y.cpu().numpy(), "L": tl.cpu().numpy(), "plan": plan}
    if gy is not None:
        gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
        plan.filter_mix_backward(dev(gy), x, g, gx, gr, gg)
        out.update(dx=gx.cpu().numpy(), dh=gr.cpu().numpy(), da=gg.cpu().numpy())
    plan.sync_status()
    return out


def channels(v, ny, J):
    off = np.concatenate([[0], np.cumsum(ny * J)])
    for u in range(ny.shape[0]):
        for j in range(J):
            yield u, j, v[off[u] + j * ny[u]:off[u] + (j + 1) * ny[u]]


CASES = [(20.0, 0, None), (math.inf, 16384, [8192]), (10.0, 16384, None), (30.0, 0, [16384]),
         (20.0, 16384, [4096])]


@pytest.mark.parametrize("eta,seg,fft_sizes", CASES)
def test_full_output_forward_matches_oracle(eta, seg, fft_sizes):
    b = full_batch()
    S = int(np.sum(b.num_sources))
    gains = np.linspace(0.5, 1.5, S).astype(np.float32)
    got = run(b, eta, gains, seg=seg, fft_sizes=fft_sizes)
    ref = oracle.forward(b, eta, alpha=gains.astype(np.float64), output_mode=1)
    assert np.array_equal(got["L"], ref["L"])
    ny = synth.output_lengths(b, 1)
    assert got["plan"].y_size == int(np.sum(ny)) * b.num_mics
    assert not np.any(np.isnan(got["y"]))
    ri = b.rir_index()
    for (u, j, g), (_, _, r) in zip(channels(got["y"], ny, b.num_mics), channels(ref["y"], ny, b.num_mics)):
        lmax = int(ref["L"][ri[u]:ri[u + 1]].max())
        end = int(b.num_samples[u]) + lmax - 1
        assert np.all(g[end:] == 0.0), f"u={u} j={j}: nonzero output past Nx + L_max - 1"
        peak = np.abs(r).max()
        rl2 = np.linalg.norm(g.astype(np.float64) - r) / np.linalg.norm(r)
        assert rl2 <= REL_L2, f"u={u} j={j}: rel L2 {rl2:.3e}"
        assert np.abs(g - r).max() <= MAX_ABS * peak


@pytest.mark.parametrize("eta,seg,bseg,fft_sizes", [(20.0, 0, 0, None), (math.inf, 16384, 16384, [8192]),
                                                    (10.0, 0, 40000, [2048, 4096])])
def test_full_output_backward_matches_oracle(eta, seg, bseg, fft_sizes):
    b = full_batch(41)
    S = int(np.sum(b.num_sources))
    gains = np.linspace(0.6, 1.3, S).astype(np.float32)
    ny = synth.output_lengths(b, 1)
    gy = synth.grad_like(42, int(np.sum(ny)) * b.num_mics)
    got = run(b, eta, gains, gy=gy, seg=seg, bseg=bseg, fft_sizes=fft_sizes)
    L = oracle.truncate_batch(b, eta)["L"]
    ref = oracle.backward(b, L, gains.astype(np.float64), gy, output_mode=1)

    grads_close(b, ref, L, dx=got["dx"], dh=got["dh"], dalpha=got["da"])


def test_full_output_prefix_is_the_same_output():
    # the first Nx samples of the full output are the "same" output of another plan
    from paper_1712_03439_gb300 import Plan
    b = full_batch(51)
    S = int(np.sum(b.num_sources))
    gains = np.linspace(0.7, 1.1, S).astype(np.float32)
    full = run(b, 20.0, gains)
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(dev(b.x), dev(b.rir), dev(gains), y)
    plan.sync_status()
    same = y.cpu().numpy()
    ny, nx = synth.output_lengths(b, 1), b.num_samples.astype(np.int64)
    for (u, j, f), (_, _, s) in zip(channels(full["y"], ny, b.num_mics), channels(same, nx, b.num_mics)):
        peak = max(np.abs(s).max(), 1e-30)
        assert np.abs(f[:nx[u]] - s).max() <= 1e-6 * peak, f"u={u} j={j}"
