"""Host-side logic without a GPU: the streaming batcher's admission, the
output-length bookkeeping and the benchmark's roofline arithmetic."""
import importlib.util
import math
import os

import numpy as np
import pytest

from paper_1712_03439_gb300 import synth
from paper_1712_03439_gb300.stream import admit, group_bytes, utterance_bytes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _utt_bytes(b, u, **kw):
    ri = b.rir_index()
    lens = b.rir_len[ri[u]:ri[u + 1]]
    return utterance_bytes(int(b.num_samples[u]), int(b.num_sources[u]), b.num_mics, int(lens.sum()),
                           int(lens.max()), **kw)


@pytest.mark.parametrize("budget_mb", [8, 32, 200])
def test_admission_covers_the_queue_in_order_within_budget(budget_mb):
    b = synth.config_stream(n_utts=60)
    budget = budget_mb << 20
    groups = admit(b, budget)
    assert [u for g in groups for u in g] == list(range(b.num_utts))
    for g in groups:
        need = group_bytes(b, g)
        # a group fits, or it is a single utterance too large for any group
        assert need <= budget or len(g) == 1
        # greedy: the next utterance would not have fitted
        if g.stop < b.num_utts:
            assert group_bytes(b, range(g.start, g.stop + 1)) > budget


def test_admission_counts_the_backward_and_the_full_output():
    b = synth.trim_rirs(synth.config_stream(n_utts=20), 5)
    fwd_only = sum(_utt_bytes(b, u, backward=False) for u in range(b.num_utts))
    both = sum(_utt_bytes(b, u) for u in range(b.num_utts))
    full = sum(_utt_bytes(b, u, output_mode=1) for u in range(b.num_utts))
    assert fwd_only < both < full
    # the full output adds J * (longest RIR - 1) samples per utterance, twice (y and grad_y)
    ri = b.rir_index()
    extra = sum(2 * 4 * b.num_mics * (int(b.rir_len[ri[u]:ri[u + 1]].max()) - 1) for u in range(b.num_utts))
    assert full - both == extra


def test_output_lengths_same_and_full():
    b = synth.trim_rirs(synth.config_stream(n_utts=12), 9)
    same = synth.output_lengths(b, 0)
    full = synth.output_lengths(b, 1)
    np.testing.assert_array_equal(same, b.num_samples)
    ri = b.rir_index()
    for u in range(b.num_utts):
        assert full[u] == b.num_samples[u] + b.rir_len[ri[u]:ri[u + 1]].max() - 1


def test_trim_rirs_keeps_a_prefix_of_each_rir():
    b = synth.config_stream(n_utts=6)
    t = synth.trim_rirs(b, 3, min_frac=0.4)
    ro, rt = b.rir_offsets(), t.rir_offsets()
    for r in range(b.num_rirs):
        n = int(t.rir_len[r])
        assert math.ceil(0.4 * b.rir_len[r]) <= n <= b.rir_len[r]
        np.testing.assert_array_equal(t.rir[rt[r]:rt[r + 1]], b.rir[ro[r]:ro[r] + n])


def test_roofline_arithmetic():
    bench = _bench()
    # 1e12 flops and 1e9 bytes in 50 ms against 80 TFLOP/s and 5000 GB/s: ALU bound
    r = bench.roofline_entry(1e12, 1e9, 50.0, 80.0, 5000.0, "measured", None)
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(20.0)
    assert r["frac"] == pytest.approx(0.25)
    assert r["hbm_side"]["achieved"] == pytest.approx(20.0)
    # the same time with 1e11 flops and 1e11 bytes: HBM bound
    r = bench.roofline_entry(1e11, 1e11, 50.0, 80.0, 5000.0, "measured", 123.0)
    assert r["bound"] == "hbm" and r["traffic"] == 123.0
    assert r["frac"] == pytest.approx(1e11 / 0.05 / 1e9 / 5000.0)
    w = {"fwd_flops": 4e10, "bwd_flops": 6e10, "fwd_bytes": 1e9, "bwd_bytes": 2e9,
         "fwd_flops_5n": 8e10, "bwd_flops_5n": 1.2e11}
    st = bench.step_roofline(w, 2.5, 80.0, 5000.0)
    assert st["t_roof_ms"] == pytest.approx(1e11 / 80e12 * 1e3)
    assert st["frac"] == pytest.approx(st["t_roof_ms"] / 2.5)
    assert st["t_roof_ms_5NlogN"] == pytest.approx(2e11 / 80e12 * 1e3)
    assert st["bound"] == "alu"


def test_algorithmic_work_counts_transforms_and_bytes():
    bench = _bench()
    b = synth.make_batch(3, [10000, 20000], [1, 2], synth.linear_pair_array(), (0.1, 0.1))
    q = {"log2_n": np.array([13, 12]), "num_blocks": np.array([3, 7])}
    L = np.full(b.num_rirs, 500)
    w = bench.algorithmic_work(b, q, L)
    J = 2
    tr = lambda m: 2.5 * (1 << m) * m
    mac = lambda m: 8.0 * ((1 << m) / 2 + 1)
    ff = 3 * ((1 + J) * tr(13) + 1 * J * mac(13)) + 7 * ((2 + J) * tr(12) + 2 * J * mac(12))
    assert w["fwd_flops"] == pytest.approx(ff)
    assert w["fwd_bytes"] == pytest.approx(4.0 * ((1 + J) * 10000 + (2 + J) * 20000))
    bf = (3 * ((2 + J) * tr(13) + 2 * J * mac(13)) + 1 * J * tr(13)
          + 7 * ((4 + J) * tr(12) + 4 * J * mac(12)) + 2 * J * tr(12))
    assert w["bwd_flops"] == pytest.approx(bf)
    assert w["fwd_flops_5n"] > w["fwd_flops"]


def test_algorithmic_work_with_the_spectrum_cache():
    # each source block is transformed once for the step: the backward does I + J transforms
    # per block and reads the kept spectra (4N bytes per source block) instead of x, which
    # the forward writes -- at every size
    bench = _bench()
    b = synth.make_batch(3, [10000, 20000], [1, 2], synth.linear_pair_array(), (0.1, 0.1))
    L = np.full(b.num_rirs, 500)
    J = 2
    tr = lambda m: 2.5 * (1 << m) * m
    mac = lambda m: 8.0 * ((1 << m) / 2 + 1)
    q = {"log2_n": np.array([13, 14]), "num_blocks": np.array([3, 2])}
    plain = bench.algorithmic_work(b, q, L)
    w = bench.algorithmic_work(b, q, L, cache=True)
    assert w["fwd_flops"] == pytest.approx(plain["fwd_flops"])
    spec = 3 * 1 * 4.0 * 8192 + 2 * 2 * 4.0 * 16384
    assert w["fwd_bytes"] == pytest.approx(plain["fwd_bytes"] + spec)
    assert w["bwd_bytes"] == pytest.approx(plain["bwd_bytes"] - 4.0 * (1 * 10000 + 2 * 20000) + spec)
    assert plain["bwd_flops"] - w["bwd_flops"] == pytest.approx(3 * 1 * tr(13) + 2 * 2 * tr(14))


def test_room_recipe_keeps_everything_inside_the_room():
    b = synth.config_stream(n_utts=40)
    geom, rir_len, rt60 = synth.room_geometry(5, b.num_sources, synth.linear_pair_array())
    assert geom.shape == (b.num_rirs, 10) and rir_len.shape == (b.num_rirs,)
    room, src, mic, refl = geom[:, :3], geom[:, 3:6], geom[:, 6:9], geom[:, 9]
    assert np.all((src > 0) & (src < room)) and np.all((mic > 0) & (mic < room))
    assert np.all((refl >= 0) & (refl < 1))
    # one room per utterance, every RIR of it ceil(RT60 fs) taps, the pair 7.1 cm apart
    ri = b.rir_index()
    for u in range(b.num_utts):
        rows = geom[ri[u]:ri[u + 1]]
        assert np.all(rows[:, :3] == rows[0, :3]) and np.all(rows[:, 9] == rows[0, 9])
        assert np.all(rir_len[ri[u]:ri[u + 1]] == math.ceil(rt60[u] * synth.FS))
        m = rows[:, 6:9].reshape(-1, b.num_mics, 3)[0]
        assert np.linalg.norm(m[0] - m[1]) == pytest.approx(0.071, abs=1e-5)


def test_excerpt_cuts_every_source_alike():
    b = synth.make_batch(3, [1000, 400, 2500], [2, 1, 3], synth.linear_pair_array(), (0.1, 0.1))
    e = b.excerpt(600)
    np.testing.assert_array_equal(e.num_samples, [600, 400, 600])
    xo, eo = b.x_offsets(), e.x_offsets()
    for s in range(int(b.num_sources.sum())):
        n = eo[s + 1] - eo[s]
        np.testing.assert_array_equal(e.x[eo[s]:eo[s + 1]], b.x[xo[s]:xo[s] + n])
    np.testing.assert_array_equal(e.rir, b.rir)
    np.testing.assert_array_equal(e.snr_db, b.snr_db)


def test_generator_and_front_end_work_counts():
    bench = _bench()
    nbytes, flops = bench.image_work(3, [100, 200, 300], 8)
    assert nbytes == 4.0 * 600 + 48.0 * 3 + 8.0
    assert flops == 6.0 * 3 * 17 ** 3
    nbytes, flops = bench.mel_work(np.array([16000, 8000]), 45, 141)
    assert nbytes == 4.0 * 24000 + 4.0 * 45 * 4 * 128
    assert flops == 141 * (512 + 2.5 * 512 * 9 + 3 * 257 + 2 * 2 * 257)
