"""Streaming workload: a queue of utterances (log-uniform 0.5-20 s, 1-4
sources, 2 mics) run in batches admitted by a memory budget.  Every utterance
is processed once, in order, within the budget, and sampled utterances of
several batches match the FP64 oracle (gains, lengths, outputs, gradients)."""
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


def close(g, r, what):
    g = g.astype(np.float64)
    peak = np.abs(r).max()
    rl2 = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
    assert rl2 <= REL_L2, f"{what}: rel L2 {rl2:.3e}"
    assert np.abs(g - r).max() <= MAX_ABS * max(peak, 1e-30), what


def test_stream_batches_cover_queue_within_budget_and_match_oracle():
    from paper_1712_03439_gb300.stream import Streamer
    b = synth.config_stream(n_utts=160)
    budget = 64 << 20
    st = Streamer(budget_bytes=budget, eta_db=20.0, backward=True)
    grads = {}

    def grad_y(sub, ny):
        g = synth.grad_like(500 + len(grads), int(ny.sum()) * sub.num_mics)
        grads[len(grads)] = g
        return g

    res = st.run(b, grad_y=grad_y)
    assert len(res.records) >= 3
    # the shape-class plan serves most batches (re-planned in place)
    assert sum(r.reshaped for r in res.records) >= len(res.records) - 1
    covered = [u for r in res.records for u in r.utts]
    assert covered == list(range(b.num_utts))
    for r in res.records:
        assert r.footprint_bytes <= budget or len(r.utts) == 1, (r.utts, r.footprint_bytes)
        assert r.wall_ms > 0 and r.device_ms > 0
    assert 0 < res.latency_ms(50) <= res.latency_ms(99)
    # sampled utterances from the first, a middle and the last batch
    for bi in (0, len(res.records) // 2, len(res.records) - 1):
        rec, out = res.records[bi], res.outputs[bi]
        sub = b.subset(rec.utts)
        k = len(rec.utts) - 1                         # last utterance of the batch
        one = sub.subset([k])
        ref = oracle.forward(one, 20.0)
        si, ri, yo, xo, ro = sub.src_index(), sub.rir_index(), sub.y_offsets(), sub.x_offsets(), sub.rir_offsets()
        np.testing.assert_allclose(out["gains"][si[k]:si[k + 1]], ref["alpha"], rtol=1e-6)
        np.testing.assert_array_equal(out["trunc_len"][ri[k]:ri[k + 1]], ref["L"].astype(np.int32))
        close(out["y"][yo[k]:yo[k + 1]], ref["y"], f"y batch {bi}")
        gref = oracle.backward(one, ref["L"], out["gains"][si[k]:si[k + 1]].astype(np.float64),
                               grads[bi][yo[k]:yo[k + 1]])
        grads_close(one, gref, ref["L"], dx=out["grad_x"][xo[si[k]]:xo[si[k + 1]]],
                    dh=out["grad_rir"][ro[ri[k]]:ro[ri[k + 1]]], dalpha=out["grad_gains"][si[k]:si[k + 1]],
                    what=f"batch {bi} ")


def test_admission_estimate_bounds_the_real_footprint():
    # the estimate the batcher admits by is an upper bound of buffers + real scratch
    from paper_1712_03439_gb300.stream import Streamer, admit, group_bytes
    b = synth.config_stream(seed=171203443 + 7, n_utts=40)
    est = group_bytes(b, range(b.num_utts))
    st = Streamer(budget_bytes=1 << 40, keep_outputs=False)
    res = st.run(b, groups=[range(b.num_utts)])
    assert res.records[0].footprint_bytes <= est
    assert len(admit(b, est)) == 1
