"""Upper-bound plans (rsim_plan_reshape) on the GPU: a plan made for a large
batch, re-planned in place for smaller batches, gives bitwise the results of a
plan made for each batch (eager and through replayed graphs); a batch beyond
the class is refused and the plan keeps its shape; only the batch shape may
change."""
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


def run(plan, b, seed, calls=1):
    S = int(b.num_sources.sum())
    x, rir, g = dev(b.x), dev(b.rir), dev(np.linspace(0.5, 1.3, S))
    gy = dev(synth.grad_like(seed, b.y_size))
    y = torch.empty(plan.y_size, device="cuda")
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(g)
    tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
    for _ in range(calls):
        plan.filter_mix(x, rir, g, y, trunc_len=tl)
        plan.filter_mix_backward(gy, x, g, gx, gr, gg)
    plan.sync_status()
    return [t.cpu().numpy() for t in (y, tl, gx, gr, gg)]


def batches():
    mics = synth.linear_pair_array()
    # the class dominates every batch below in utterances, sources, samples, segments and taps
    big = synth.make_batch(501, [70000, 33000, 50000, 12000, 9000, 1000], [4, 2, 3, 1, 3, 2], mics, (0.1, 0.4))
    small = [synth.make_batch(502, [9000, 41000], [3, 2], mics, (0.1, 0.3)),
             synth.make_batch(503, [66000], [4], mics, (0.2, 0.4)),
             synth.make_batch(504, [1, 700, 3000, 20011, 5000], [1, 2, 1, 1, 2], mics, (0.1, 0.2))]
    return big, small


@pytest.mark.parametrize("graphs", [False, True])
def test_reshaped_plan_equals_fresh_plans(graphs):
    from paper_1712_03439_gb300 import Plan
    big, small = batches()
    plan = Plan.for_batch(big, eta_db=20.0, gain_mode=1, graphs=graphs)
    ref_big = run(Plan.for_batch(big, eta_db=20.0, gain_mode=1, graphs=False), big, 7)
    for a, c in zip(run(plan, big, 7, calls=2), ref_big):
        np.testing.assert_array_equal(a, c)
    for k, b in enumerate(small + [big]):
        plan.reshape_for(b)
        assert plan.U == b.num_utts and plan.x_size == b.x.size
        got = run(plan, b, 10 + k, calls=2)            # with graphs: capture, then replay
        ref = run(Plan.for_batch(b, eta_db=20.0, gain_mode=1, graphs=False), b, 10 + k)
        for a, c in zip(got, ref):
            np.testing.assert_array_equal(a, c)


def test_batch_beyond_the_class_is_refused_and_the_plan_keeps_its_shape():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    big, small = batches()
    plan = Plan.for_batch(small[0], eta_db=20.0, gain_mode=1)
    before = run(plan, small[0], 21)
    with pytest.raises(RsimError) as e:
        plan.reshape_for(big)                          # more samples than the class holds
    assert e.value.status == 2
    assert plan.U == small[0].num_utts
    for a, c in zip(run(plan, small[0], 21), before):
        np.testing.assert_array_equal(a, c)


def test_only_the_batch_shape_may_change():
    from paper_1712_03439_gb300 import Plan
    from paper_1712_03439_gb300._lib import RsimError
    big, small = batches()
    plan = Plan.for_batch(big, eta_db=20.0, gain_mode=1)
    plan._fixed = dict(plan._fixed, eta_db=10.0)
    with pytest.raises(RsimError) as e:
        plan.reshape_for(small[0])
    assert e.value.status == 1
