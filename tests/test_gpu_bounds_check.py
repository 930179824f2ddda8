"""The bounds-checked build on the GPU: a forward and backward through
librsim_checked.so (every kernel store checked against its buffer) latch no
error and give bitwise the release library's results."""
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
    build.build_checked()


def _run(b, gains, gy, sizes, eta=20.0, long_rirs=False):
    from paper_1712_03439_gb300 import Plan
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    plan = Plan.for_batch(b, eta_db=eta, gain_mode=1, fft_sizes=sizes, long_rirs=long_rirs)
    x, rir, g = dev(b.x), dev(b.rir), dev(gains)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(x, rir, g, y)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
    plan.filter_mix_backward(dev(gy), x, g, gx, gr, gg)
    plan.sync_status()                     # raises if a checked store latched
    out = [t.cpu().numpy() for t in (y, gx, gr, gg)]
    plan.close()
    return out


@pytest.mark.parametrize("sizes,J", [(None, 2), ([2048], 3), ([16384], 2)])
def test_checked_build_is_clean_and_equal(sizes, J):
    from paper_1712_03439_gb300 import _lib, build
    mics = synth.linear_pair_array() if J == 2 else synth.circular_array(J, 0.05)
    b = synth.make_batch(401, [900, 20011, 50000], [2, 3, 5], mics, (0.1, 0.2))
    S = int(b.num_sources.sum())
    gains = np.linspace(0.5, 1.3, S).astype(np.float32)
    gy = synth.grad_like(402, b.y_size)
    release = _run(b, gains, gy, sizes)
    saved = _lib._lib
    _lib._lib = _lib.load(build.CHECKED_LIB_PATH)
    try:
        checked = _run(b, gains, gy, sizes)
    finally:
        _lib._lib = saved
    for a, c in zip(release, checked):
        np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("eta", [30.0, float("inf")])
def test_checked_build_with_a_partitioned_path_is_clean_and_equal(eta):
    # one utterance whose kept RIRs exceed one block of N = 16384 (its partitioned path:
    # the copies onto that plan and back are checked too) beside one that fits
    from paper_1712_03439_gb300 import _lib, build
    mics = synth.linear_pair_array()
    a = synth.make_batch(411, [9000], [2], mics, (2.2, 2.4))
    c = synth.make_batch(412, [700], [1], mics, (0.2, 0.3))
    b = synth.Batch(2, np.concatenate([a.num_sources, c.num_sources]), np.concatenate([a.num_samples, c.num_samples]),
                    np.concatenate([a.rir_len, c.rir_len]), np.concatenate([a.x, c.x]),
                    np.concatenate([a.rir, c.rir]), np.concatenate([a.snr_db, c.snr_db]))
    S = int(b.num_sources.sum())
    gains = np.linspace(0.5, 1.3, S).astype(np.float32)
    gy = synth.grad_like(413, b.y_size)
    release = _run(b, gains, gy, None, eta=eta, long_rirs=True)
    saved = _lib._lib
    _lib._lib = _lib.load(build.CHECKED_LIB_PATH)
    try:
        checked = _run(b, gains, gy, None, eta=eta, long_rirs=True)
    finally:
        _lib._lib = saved
    for x, y in zip(release, checked):
        np.testing.assert_array_equal(x, y)
