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


def _run(b, gains, gy, sizes):
    from paper_1712_03439_gb300 import Plan
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, fft_sizes=sizes)
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
