"""Image-method RIRs (Eq. 1): CUDA path vs the FP64 oracle.

The oracle lands each image at ceil(t), t = d fs / c0 evaluated in FP64.  The
kernel evaluates the same real number in FP32, so an image whose t lies within
a few FP32 rounding errors of an integer m may land on m or on m + 1: both
are readings of Eq. 1.  For every other image the tap must be the oracle's.
So each RIR is compared against the oracle's images with the near-integer
ones placed where the kernel put them (the placement of each group of such
images that best explains the kernel's taps); every remaining tap, the
support (amplitudes are positive, so colliding images never cancel) and the
values must then match: per RIR a relative L2 error <= 1e-5 and a max-abs
error <= 1e-5 x its peak, the tolerance of the filter-and-mix path (the
kernel's FP32 amplitudes and FP32 sums where images collide against FP64).
"""
import math

import numpy as np
import pytest

import oracle
from image_checks import _near_threshold, _valid_cut, check_rir, settle
from paper_1712_03439_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-5
WINDOW = 11264        # taps per kernel window (lengths around it are covered)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03439_gb300 import build
    build.build()


def gpu_rirs(geom, lens, order=8, fs=16000.0, c0=343.0, max_len=None, off=None):
    from paper_1712_03439_gb300 import image_rirs
    geom = np.ascontiguousarray(np.asarray(geom, dtype=np.float32).reshape(-1, 10))
    if off is None:
        off = np.concatenate([[0], np.cumsum(np.asarray(lens, dtype=np.int64))])
    total = int(max(off.max(), 0))
    rir = torch.full((max(total, 1),), float("nan"), device="cuda")   # every tap must be written
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    image_rirs(torch.from_numpy(geom).cuda(), torch.from_numpy(np.asarray(off, np.int64)).cuda(),
               int(max(lens) if max_len is None else max_len) if len(lens) else 0, rir, order=order,
               fs=fs, c0=c0, status=status)
    torch.cuda.synchronize()
    return rir.cpu().numpy()[:total], int(status.item()), off


def random_rooms(seed, n, lens=None):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        room = rng.uniform([2.0, 2.0, 2.0], [12.0, 9.0, 6.0])
        rows.append(np.concatenate([room, rng.uniform(0.05, 0.95, 3) * room,
                                    rng.uniform(0.05, 0.95, 3) * room, [rng.uniform(0.1, 0.95)]]))
    geom = np.asarray(rows, dtype=np.float32)
    if lens is None:
        lens = rng.integers(1, 12000, n)
    return geom, np.asarray(lens, dtype=np.int64)


def compare_all(geom, lens, order, **kw):
    """Every RIR against the oracle's, near-integer images settled.  Returns
    (kernel RIRs, settled oracle RIRs, near-integer images seen)."""
    fs, c0 = kw.get("fs", 16000.0), kw.get("c0", 343.0)
    got, status, off = gpu_rirs(geom, lens, order=order, **kw)
    assert status == 0
    plain, valid = oracle.image_rirs(geom, lens, order=order, fs=fs, c0=c0)
    assert valid.all()
    want = np.zeros_like(plain)
    ties = 0
    for r in range(len(lens)):
        w, n = settle(got[off[r]:off[r + 1]], geom[r], int(lens[r]), order, fs, c0)
        ties += n
        # the settled RIR differs from the oracle's only on near-integer images
        if n == 0:
            np.testing.assert_allclose(w, plain[off[r]:off[r + 1]], rtol=1e-13, atol=0)
        want[off[r]:off[r + 1]] = w
        check_rir(got[off[r]:off[r + 1]], w, f"RIR {r} (order {order})")
    return got, want, ties


@pytest.mark.parametrize("order", [0, 1, 3, 8, 12])
def test_random_rooms_match_oracle(order):
    lens = [1, 2, 700, 5000, WINDOW - 1, WINDOW, WINDOW + 1, 2 * WINDOW + 3, 11111, 9000, 4321, 3]
    geom, lens = random_rooms(100 + order, len(lens), lens)
    compare_all(geom, lens, order)


def test_long_rirs_span_several_windows():
    # a large room at a high order: images land over more than 3 windows
    geom = np.array([[30.0, 25.0, 12.0, 4.1, 7.3, 2.2, 20.5, 3.3, 9.1, 0.9],
                     [18.0, 11.0, 7.0, 17.0, 1.0, 6.5, 0.5, 10.0, 0.25, 0.7]], np.float32)
    lst = oracle.image_list(geom[0, :3], geom[0, 3:6], geom[0, 6:9], geom[0, 9], order=24)
    n_h = int(lst["delay"].max()) + 1
    assert n_h > 3 * WINDOW
    got, want, _ = compare_all(geom, [n_h, 50001], 24)
    assert np.count_nonzero(want[:n_h][3 * WINDOW:]) > 0


def test_other_rates_and_speeds():
    geom, lens = random_rooms(7, 8)
    compare_all(geom, lens, 8, fs=48000.0, c0=340.0)
    compare_all(geom, lens, 8, fs=8000.0, c0=343.0)


def test_exact_delay_and_direct_path_only():
    # fs / c0 = 64: a 0.5 m path is 32 samples exactly, 133/256 m is 33.25 -> 34
    geom = np.array([[4, 4, 4, 1, 1, 1, 1.5, 1, 1, 0.0],
                     [4, 4, 4, 1, 1, 1, 1 + 133 / 256, 1, 1, 0.0]], np.float32)
    got, status, off = gpu_rirs(geom, [64, 64], order=8, fs=16000.0, c0=250.0)
    assert status == 0
    assert np.flatnonzero(got[:64]).tolist() == [32]
    assert got[32] == pytest.approx(2.0, rel=1e-6)
    assert np.flatnonzero(got[64:]).tolist() == [34]
    assert got[64 + 34] == pytest.approx(256 / 133, rel=1e-6)


def test_home_rooms_workload_matches_oracle():
    """The benchmark's rooms workload (256 utterances, about 1250 RIRs of
    1.6k-14.4k taps) at the paper's 17^3 virtual rooms, every RIR compared."""
    b, geom = synth.config_home_rooms()
    _, _, ties = compare_all(geom, b.rir_len.astype(np.int64), 8)
    # about 6 million images: some travel times sit near an integer
    assert ties > 0


def test_invalid_rirs_and_edge_cases():
    geom, lens = random_rooms(11, 6, [300, 0, 1, 250, 400, 120])
    geom[3, 9] = 1.0                      # r = 1: invalid
    geom[4, 6:9] = geom[4, 3:6]           # microphone at the source: an image at distance 0
    got, status, off = gpu_rirs(geom, lens, order=8)
    assert status == 1
    want, valid = oracle.image_rirs(geom, lens, order=8)
    assert valid.tolist() == [True, True, True, False, False, True]
    for r in range(6):
        seg = got[off[r]:off[r + 1]]
        if valid[r]:
            check_rir(seg, settle(seg, geom[r], int(lens[r]), 8, 16000.0, 343.0)[0], f"RIR {r}")
        else:
            assert seg.shape[0] == lens[r] and not seg.any()
    # length 1: the earliest possible delay is 1, so the tap is zero
    assert got[off[2]] == 0.0


def test_max_len_only_sizes_the_grid():
    geom, lens = random_rooms(12, 4, [40000, 100, 20000, 5])
    got, status, off = gpu_rirs(geom, lens, order=8, max_len=10)
    assert status == 0
    for r in range(4):
        seg = got[off[r]:off[r + 1]]
        check_rir(seg, settle(seg, geom[r], int(lens[r]), 8, 16000.0, 343.0)[0], f"RIR {r}")


def test_bad_length_is_flagged_and_not_written():
    geom, _ = random_rooms(13, 2, [100, 1])
    off = np.array([0, 100, 40], np.int64)           # RIR 1 has a negative length
    got, status, _ = gpu_rirs(geom, [100, 1], order=8, off=off)
    assert status == 2
    check_rir(got[:100], settle(got[:100], geom[0], 100, 8, 16000.0, 343.0)[0], "RIR 0")


def test_empty_batch_resets_status():
    from paper_1712_03439_gb300 import image_rirs
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    image_rirs(torch.zeros((0, 10), device="cuda"), torch.zeros(1, dtype=torch.int64, device="cuda"), 0,
               torch.zeros(1, device="cuda"), status=status)
    assert int(status.item()) == 0


def test_graph_replay_matches_eager():
    from paper_1712_03439_gb300 import image_rirs
    geom, lens = random_rooms(14, 5)
    off = np.concatenate([[0], np.cumsum(lens)])
    g = torch.from_numpy(geom).cuda()
    o = torch.from_numpy(off).cuda()
    eager = torch.zeros(int(off[-1]), device="cuda")
    image_rirs(g, o, int(lens.max()), eager)
    out = torch.zeros_like(eager)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            image_rirs(g, o, int(lens.max()), out, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    # colliding images are summed by shared-memory atomics, so the two runs may
    # differ in the last bits: each is compared with the oracle
    e, r = eager.cpu().numpy(), out.cpu().numpy()
    for k in range(len(lens)):
        for name, v in (("replayed", r), ("eager", e)):
            seg = v[off[k]:off[k + 1]]
            check_rir(seg, settle(seg, geom[k], int(lens[k]), 8, 16000.0, 343.0)[0], f"{name} RIR {k}")


def test_generated_rirs_feed_the_mix():
    """Image RIRs made on the device go straight into filter_mix; the oracle
    takes the same rooms' images (near-integer ones settled as in the RIR
    tests), cuts them and mixes.  Cut-off lengths are exact wherever no tap
    sits within 1e-5 of the threshold; where one does, the kernel's length
    must be a valid cut of the oracle's RIR, and the mix is compared with the
    oracle at the kernel's lengths, so it is compared in every case."""
    import dataclasses
    from paper_1712_03439_gb300 import Plan, image_rirs
    # RT60 up to 0.7 s keeps every untruncated RIR within the largest FFT size's reach
    b = synth.config_home(seed=synth.SEED_BASE + 50, n_utts=6)
    geom, rir_len, _ = synth.room_geometry(synth.SEED_BASE + 51, b.num_sources, synth.linear_pair_array(),
                                           rt60_range=(0.1, 0.7))
    b = dataclasses.replace(b, rir_len=rir_len, rir=np.zeros(int(rir_len.sum()), np.float32))
    lens = b.rir_len.astype(np.int64)
    off = np.concatenate([[0], np.cumsum(lens)])
    rng = np.random.default_rng(5)
    alpha = np.where(np.arange(int(b.num_sources.sum())) == 0, 1.0, rng.uniform(0.2, 1.0,
                     int(b.num_sources.sum()))).astype(np.float32)
    compared = 0
    for eta in (math.inf, 20.0):
        rir = torch.empty(int(off[-1]), device="cuda")
        image_rirs(torch.from_numpy(geom).cuda(), torch.from_numpy(off).cuda(), int(lens.max()), rir)
        h_gpu = rir.cpu().numpy()
        h_or = np.concatenate([settle(h_gpu[off[r]:off[r + 1]], geom[r], int(lens[r]), 8, 16000.0, 343.0)[0]
                               for r in range(len(lens))])
        bo = dataclasses.replace(b, rir=h_or.astype(np.float32))
        plan = Plan.for_batch(b, eta_db=eta, gain_mode=1)
        x = torch.from_numpy(b.x).cuda()
        y = torch.empty(plan.y_size, device="cuda")
        tl = torch.empty(plan.R, dtype=torch.int32, device="cuda")
        plan.filter_mix(x, rir, torch.from_numpy(alpha).cuda(), y, trunc_len=tl)
        plan.sync_status()
        L = tl.cpu().numpy()
        L_or = oracle.truncate_batch(bo, eta)["L"]
        for r in range(len(lens)):
            h = h_or[off[r]:off[r + 1]]
            if _near_threshold(h, eta):
                assert _valid_cut(h, int(L[r]), eta), f"RIR {r}: cut {L[r]} is no reading of Eq. 8"
            else:
                assert L[r] == L_or[r], f"RIR {r}: cut {L[r]} vs {L_or[r]}"
        want = {"y": oracle.forward_with_lengths(bo, L.astype(np.int64), alpha.astype(np.float64))}
        got = y.cpu().numpy().astype(np.float64)
        yo = b.y_offsets()
        for u in range(b.num_utts):
            for j in range(b.num_mics):
                n = int(b.num_samples[u])
                s = slice(int(yo[u]) + j * n, int(yo[u]) + (j + 1) * n)
                err = got[s] - want["y"][s]
                assert np.linalg.norm(err) <= REL_L2 * np.linalg.norm(want["y"][s])
                assert np.max(np.abs(err)) <= MAX_ABS * np.max(np.abs(want["y"][s]))
                compared += 1
    assert compared == 2 * b.num_utts * b.num_mics
