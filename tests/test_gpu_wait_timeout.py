"""Bounded waits: when a bulk copy a kernel waits for never completes, the wait
runs out (about half a second), the kernel latches an error bit and stops, the
host reports RSIM_E_DEVICE, and the context stays usable.

The copy is withheld on the host side of the test: a plan made while
RSIM_TEST_WITHHOLD_BULK_COPY=1 tells the backward's barriers to expect the
bytes but issues no copy.  No fault, trap or endless loop is involved."""
import os
import time

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


def _run(plan, b, gains):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, rir, g = dev(b.x), dev(b.rir), dev(gains)
    y = torch.empty(plan.y_size, device="cuda")
    plan.filter_mix(x, rir, g, y)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
    plan.filter_mix_backward(dev(synth.grad_like(3, b.y_size)), x, g, gx, gr, gg)
    return gx


def test_withheld_bulk_copy_times_out_and_is_reported():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    b = synth.make_batch(77, [20000, 9000], [2, 1], synth.linear_pair_array(), (0.1, 0.2))
    gains = np.ones(int(b.num_sources.sum()), np.float32)
    os.environ["RSIM_TEST_WITHHOLD_BULK_COPY"] = "1"
    try:
        plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, fft_sizes=[8192], graphs=False)
    finally:
        del os.environ["RSIM_TEST_WITHHOLD_BULK_COPY"]
    t0 = time.perf_counter()
    _run(plan, b, gains)
    with pytest.raises(RsimError) as e:
        plan.sync_status()
    dt = time.perf_counter() - t0
    assert e.value.status == 5 and "bounded wait" in str(e.value)
    assert dt < 30.0
    # the context is still usable: a normal plan runs and reports success
    plan2 = Plan.for_batch(b, eta_db=20.0, gain_mode=1, fft_sizes=[8192], graphs=False)
    gx = _run(plan2, b, gains)
    plan2.sync_status()
    assert torch.isfinite(gx).all()
