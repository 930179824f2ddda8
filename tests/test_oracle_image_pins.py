"""Pins of the oracle's image-method RIR (Eq. 1) against facts that do not
come from the oracle itself:

* the image lattice built literally, by mirroring the room across one wall at
  a time (the construction Sec. 2 describes), gives every image position and
  its reflection count;
* the paper's count of 17 x 17 x 17 = 4913 virtual rooms;
* Eq. 1's ceiling delay, the ceiling of the FP64 travel time d fs / c0 from
  that lattice, and exact on geometries where d fs / c0 is an exact number;
* closed forms: r = 0 leaves a single delta 1/d at ceil(d fs / c0);
* reciprocity (source and microphone swapped give the same response) on
  geometries whose coordinates are exact in FP32;
* truncating the RIR to n_h drops exactly the images at n_h or later.
"""
import math
from collections import deque

import numpy as np
import pytest

import oracle

# coordinates with few bits, so that every sum and product of positions is exact
DYADIC_ROOM = (4.0, 3.5, 2.75)
DYADIC_SRC = (1.25, 2.0, 0.75)
DYADIC_MIC = (2.5, 1.125, 1.5)
GENERIC_ROOM = (6.37, 4.91, 3.05)
GENERIC_SRC = (1.73, 3.12, 1.41)
GENERIC_MIC = (4.02, 2.26, 1.19)


def _f32(v):
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def mirrored_lattice(room, src, order):
    """Image of the source in every virtual room (a, b, c), |a|,|b|,|c| <= order,
    by breadth-first mirroring: crossing from room a to a + 1 along an axis
    reflects the point across the wall plane at (a + 1) L, crossing to a - 1
    reflects it across the plane at a L.  Returns {(a, b, c): (point, walls)}."""
    room = _f32(room)
    start = (0, 0, 0)
    seen = {start: (_f32(src), 0)}
    todo = deque([start])
    while todo:
        key = todo.popleft()
        p, walls = seen[key]
        for axis in range(3):
            for step in (1, -1):
                nxt = list(key)
                nxt[axis] += step
                nxt = tuple(nxt)
                if abs(nxt[axis]) > order or nxt in seen:
                    continue
                plane = (key[axis] + 1) * room[axis] if step == 1 else key[axis] * room[axis]
                q = p.copy()
                q[axis] = 2.0 * plane - p[axis]
                seen[nxt] = (q, walls + 1)
                todo.append(nxt)
    return seen


def _rooms(order):
    r = range(-order, order + 1)
    return [(a, b, c) for a in r for b in r for c in r]


@pytest.mark.parametrize("geom", ["dyadic", "generic"])
def test_image_positions_and_reflections_match_mirroring(geom):
    room, src, mic = (DYADIC_ROOM, DYADIC_SRC, DYADIC_MIC) if geom == "dyadic" else \
        (GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC)
    order = 3
    lat = mirrored_lattice(room, src, order)
    lst = oracle.image_list(room, src, mic, 0.8, order=order)
    assert len(lat) == len(lst["g"]) == (2 * order + 1) ** 3
    for v, key in enumerate(_rooms(order)):
        p, walls = lat[key]
        if geom == "dyadic":
            np.testing.assert_array_equal(lst["pos"][v], p)
        else:
            np.testing.assert_allclose(lst["pos"][v], p, rtol=0, atol=1e-12)
        assert lst["g"][v] == walls


@pytest.mark.parametrize("fs,c0", [(16000.0, 343.0), (48000.0, 340.0)])
def test_delays_are_ceilings_of_the_travel_time(fs, c0):
    room, src, mic = GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC
    order = 8
    lat = mirrored_lattice(room, src, order)
    lst = oracle.image_list(room, src, mic, 0.6, order=order, fs=fs, c0=c0)
    m = _f32(mic)
    t = np.array([np.linalg.norm(lat[k][0] - m) * _f32([fs])[0] / _f32([c0])[0] for k in _rooms(order)])
    # the oracle's FP64 travel time is the lattice's (up to FP64 rounding of two
    # different constructions) and its delay is that travel time's ceiling
    np.testing.assert_allclose(lst["travel"], t, rtol=1e-13, atol=0)
    d = lst["delay"]
    exact = d == np.ceil(t)
    assert np.all(exact | (np.abs(t - np.round(t)) <= 1e-9 * t))
    assert exact.mean() > 0.9999


def test_amplitudes_are_reflection_power_over_distance():
    room, src, mic = GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC
    order, refl = 4, 0.73
    lat = mirrored_lattice(room, src, order)
    lst = oracle.image_list(room, src, mic, refl, order=order)
    m = _f32(mic)
    r32 = _f32([refl])[0]
    want = np.array([r32 ** lat[k][1] / np.linalg.norm(lat[k][0] - m) for k in _rooms(order)])
    np.testing.assert_allclose(lst["amp"], want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("order", [0, 1, 2, 8])
def test_every_virtual_room_lands_when_the_rir_is_long_enough(order):
    lst = oracle.image_list(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.5, order=order)
    n_h = int(lst["delay"].max()) + 1
    h, landed = oracle.image_rir(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.5, n_h, order=order)
    # 17 x 17 x 17 = 4913 virtual rooms at the paper's order 8
    assert landed == (2 * order + 1) ** 3
    if order == 8:
        assert landed == 4913
    # the response is the sum of the images' deltas
    want = np.zeros(n_h)
    np.add.at(want, lst["delay"], lst["amp"])
    np.testing.assert_allclose(h, want, rtol=1e-13, atol=0)
    assert h.sum() == pytest.approx(lst["amp"].sum(), rel=1e-12)


def test_zero_reflection_leaves_the_direct_path():
    # fs / c0 = 64 and a 0.5 m direct path: d fs / c0 = 32 exactly, ceil(32) = 32
    h, landed = oracle.image_rir((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (1.5, 1.0, 1.0), 0.0, 200,
                                 fs=16000.0, c0=250.0)
    want = np.zeros(200)
    want[32] = 2.0
    np.testing.assert_array_equal(h, want)
    assert landed > 1   # the reflected images land too, with amplitude 0^g = 0


def test_delay_rounds_up_not_to_nearest():
    # d = 133/256 m at fs / c0 = 64: d fs / c0 = 33.25, so the delay is 34
    d = 133.0 / 256.0
    h, _ = oracle.image_rir((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (1.0 + d, 1.0, 1.0), 0.0, 64,
                            fs=16000.0, c0=250.0)
    assert np.flatnonzero(h).tolist() == [34]
    assert h[34] == pytest.approx(1.0 / d, rel=1e-15)


def test_source_and_microphone_are_interchangeable():
    a, _ = oracle.image_rir(DYADIC_ROOM, DYADIC_SRC, DYADIC_MIC, 0.7, 4000)
    b, _ = oracle.image_rir(DYADIC_ROOM, DYADIC_MIC, DYADIC_SRC, 0.7, 4000)
    assert np.count_nonzero(a) > 100
    np.testing.assert_array_equal(np.flatnonzero(a), np.flatnonzero(b))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_short_rir_is_a_prefix_of_the_long_one():
    lst = oracle.image_list(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.8)
    long_h, long_n = oracle.image_rir(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.8, int(lst["delay"].max()) + 1)
    # cut right after an image: that image stays, every later one goes
    cut = int(np.sort(lst["delay"])[len(lst["delay"]) // 3]) + 1
    short_h, short_n = oracle.image_rir(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.8, cut)
    np.testing.assert_array_equal(short_h, long_h[:cut])
    assert short_h[cut - 1] != 0.0
    assert short_n == int(np.sum(lst["delay"] < cut)) < long_n


def test_batch_form_matches_single_calls():
    rng = np.random.default_rng(7)
    rows, lens = [], []
    for _ in range(6):
        room = rng.uniform(3, 8, 3)
        src, mic = rng.uniform(0.2, 0.8, 3) * room, rng.uniform(0.2, 0.8, 3) * room
        rows.append(np.concatenate([room, src, mic, [rng.uniform(0.3, 0.9)]]))
        lens.append(int(rng.integers(50, 3000)))
    rows[3][9] = 1.0                 # invalid: r must be below 1
    geom = np.array(rows, dtype=np.float32)
    h, valid = oracle.image_rirs(geom, lens, order=3)
    assert valid.tolist() == [True, True, True, False, True, True]
    off = np.concatenate([[0], np.cumsum(lens)])
    for r in range(6):
        seg = h[off[r]:off[r + 1]]
        if valid[r]:
            g = geom[r]
            want, _ = oracle.image_rir(g[:3], g[3:6], g[6:9], g[9], lens[r], order=3)
            np.testing.assert_array_equal(seg, want)
        else:
            assert not seg.any()


@pytest.mark.parametrize("room,src,mic,refl", [
    ((4.0, 4.0, 4.0), (0.0, 1.0, 1.0), (2.0, 2.0, 2.0), 0.5),   # source on a wall
    ((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (2.0, 4.0, 2.0), 0.5),   # microphone on a wall
    ((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.5),   # source at the microphone
    ((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 1.0),   # r = 1
    ((4.0, 4.0, 4.0), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), -0.1),  # r < 0
    ((4.0, -4.0, 4.0), (1.0, 1.0, 1.0), (2.0, 2.0, 2.0), 0.5),  # negative room size
])
def test_invalid_geometry_is_rejected(room, src, mic, refl):
    with pytest.raises(oracle.OracleError):
        oracle.image_rir(room, src, mic, refl, 100)


def test_empty_rir():
    h, landed = oracle.image_rir(GENERIC_ROOM, GENERIC_SRC, GENERIC_MIC, 0.5, 0)
    assert h.size == 0 and landed == 0
