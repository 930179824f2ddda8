"""The spectrum cache: the backward reading the source half spectra the forward
kept (instead of transforming each block again).  Up to N = 8192 the forward and
the backward transform a block with the same arithmetic, so the results are
bitwise those of the plan without the cache -- with several microphone groups,
per-(i, j) gains, replayed graphs and a partitioned path.  At N = 16384 the two
kernels use different thread shapes (16 and 8 values per thread), so the cached
spectra round differently: the forward output is still bitwise the same, the
gradients agree within the parity tolerance (relative L2 and max-abs 1e-5)."""
import math

import numpy as np
import pytest

from paper_1712_03439_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run(b, cache, gain_mode, fft_sizes, graphs, eta=20.0):
    from paper_1712_03439_gb300 import Plan
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=gain_mode, fft_sizes=fft_sizes, graphs=graphs,
                          spectrum_cache=cache)
    x, rir = dev(b.x), dev(b.rir)
    if gain_mode == 2:
        gains = dev(np.random.default_rng(5).uniform(-1.2, 1.2, plan.R))
    else:
        gains = torch.empty(plan.S, device="cuda")
    y = torch.empty(plan.y_size, device="cuda")
    gy = dev(synth.grad_like(6, plan.y_size))
    gx, gr = torch.empty_like(x), torch.empty_like(rir)
    gg = torch.empty(plan.G, device="cuda")
    snr = dev(b.snr_db) if gain_mode == 0 else None
    for _ in range(2):                         # with graphs the second pair replays them
        plan.filter_mix(x, rir, gains, y, snr_db=snr)
        plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
    plan.sync_status()
    out = [t.cpu().numpy() for t in (y, gains, gx, gr, gg)]
    plan.close()
    return out


def compare(on, off, exact):
    for name, a, c in zip(("y", "gains", "dx", "dh", "dalpha"), on, off):
        if exact or name in ("y", "gains"):
            np.testing.assert_array_equal(a, c, err_msg=name)
        else:
            d = a.astype(np.float64) - c
            assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(c), name
            assert np.max(np.abs(d)) <= 1e-5 * np.max(np.abs(c)), name


@pytest.mark.parametrize("fft_sizes,J,gain_mode,graphs", [
    ([2048], 2, 0, True), ([4096], 3, 0, False), ([8192], 2, 2, True), (None, 3, 0, True), ([16384], 2, 0, True),
    ([16384], 3, 2, False),
])
def test_cached_spectra_give_the_same_results(fft_sizes, J, gain_mode, graphs):
    mics = synth.linear_pair_array() if J == 2 else synth.circular_array(J, 0.05)
    b = synth.make_batch(77 + J, [900, 20011, 50000, 7000], [2, 3, 1, 4], mics, (0.1, 0.3))
    on = run(b, True, gain_mode, fft_sizes, graphs)
    off = run(b, False, gain_mode, fft_sizes, graphs)
    compare(on, off, exact=fft_sizes is not None and max(fft_sizes) <= 8192)


def test_cached_spectra_with_a_partitioned_path():
    # parts of N = 16384 for the long RIRs: within the tolerance, not bitwise
    b = synth.trim_rirs(synth.make_batch(88, [700, 20011], [2, 3], synth.linear_pair_array(), (0.9, 1.2)), 89,
                        min_frac=0.5)
    on = run(b, True, 0, None, True, eta=math.inf)
    off = run(b, False, 0, None, True, eta=math.inf)
    compare(on, off, exact=False)


def test_cached_spectra_at_8192_with_a_partitioned_path():
    # the largest size 8192: every plan and sub-plan transforms alike, results bitwise
    b = synth.trim_rirs(synth.make_batch(90, [700, 20011], [2, 3], synth.linear_pair_array(), (0.5, 0.6)), 91,
                        min_frac=0.5)
    on = run(b, True, 0, [2048, 4096, 8192], True, eta=math.inf)
    off = run(b, False, 0, [2048, 4096, 8192], True, eta=math.inf)
    compare(on, off, exact=True)


def test_cache_memory_is_within_its_stated_bound():
    # at most 16 bytes per source sample (plus one block of the largest size per source,
    # rounded to 256 bytes): the plan's scratch grows by no more than that
    from paper_1712_03439_gb300 import Plan
    b = synth.make_batch(99, [900, 20011, 50000], [2, 3, 1], synth.linear_pair_array(), (0.1, 0.3))
    on = Plan.for_batch(b, spectrum_cache=True)
    off = Plan.for_batch(b, spectrum_cache=False)
    S = int(b.num_sources.sum())
    per_src = np.repeat(b.num_samples, b.num_sources)
    bound = int(np.sum((16 * per_src + 4 * 16384 + 255) // 256 * 256)) + 8 * (S + 1) + 2 * 256
    grown = on.scratch_bytes - off.scratch_bytes
    assert 16 * per_src.sum() <= grown <= bound
    on.close()
    off.close()

