"""Comparisons of generated image-method RIRs (Eq. 1) with the FP64 oracle,
shared by the GPU tests of the standalone generator and of the fused path.

The oracle lands each image at ceil(t), t = d fs / c0 evaluated in FP64; a
kernel evaluating the same real number in FP32 may land an image whose t lies
within a few FP32 rounding errors of an integer m on m or on m + 1, both
readings of Eq. 1.  settle() returns the oracle's RIR with each such image on
the tap that explains the kernel's output; every other image must be on the
oracle's tap.  Values: per RIR a relative L2 error <= 1e-5 and a max-abs error
<= 1e-5 x its peak.
"""
import math

import numpy as np

import oracle

REL_L2 = 1e-5
MAX_ABS = 1e-5


def _room_indices(order):
    r = np.arange(-order, order + 1)
    a, b, c = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], 1)      # (a, b, c), c fastest


U32 = 2.0 ** -24        # FP32 unit roundoff


def tie_bound(geom_row, order, fs, c0):
    """Per image, a bound (twice a first-order worst case) on how far an FP32
    evaluation of t = d fs / c0 may sit from the FP64 value: each offset to
    the microphone carries at most three roundings of numbers no larger than
    (|a| + 2) L along its axis; the squares, their sum, the square root, the
    rate and the product add at most 6 relative roundings of t."""
    room = np.asarray(geom_row[:3], np.float64)
    idx = np.abs(_room_indices(order))
    rate = float(np.float32(fs)) / float(np.float32(c0))
    de = 3 * U32 * ((idx + 2) * room).sum(1)
    return de, rate


def _group_score(choice_taps, amps, g64, base, base_cnt, lo, hi, n_h):
    """(support mismatches, absolute residual) on taps [lo, hi) for images of
    amplitude amps placed on choice_taps."""
    w = base[lo:hi].copy()
    c = base_cnt[lo:hi].copy()
    for p, a in zip(choice_taps, amps):
        if p < n_h:
            w[p - lo] += a
            c[p - lo] += 1
    return int(np.sum((c > 0) != (g64[lo:hi] != 0))), float(np.sum(np.abs(g64[lo:hi] - w)))


def settle(got, geom_row, n_h, order, fs, c0):
    """The oracle's RIR with every near-integer image on the tap, of its two
    readings (m or m + 1 for t near the integer m), that explains the
    kernel's output.  Near-integer images whose readings share a tap form a
    group; each group takes the placement with the fewest taps whose support
    differs from the kernel's, then the smallest absolute residual on its
    taps: by trying every placement for groups of up to 12 images, by moving
    one or two images at a time from the FP64 readings until nothing improves
    for longer chains.  Returns (want, near-integer images)."""
    lst = oracle.image_list(geom_row[:3], geom_row[3:6], geom_row[6:9], geom_row[9], order=order, fs=fs, c0=c0)
    t, amp, d = lst["travel"], lst["amp"], lst["delay"]
    de, rate = tie_bound(geom_row, order, fs, c0)
    bound = 2.0 * (rate * de + 6 * U32 * t)
    m = np.round(t).astype(np.int64)
    amb = (np.abs(t - m) <= bound) & (m < n_h)
    sure = ~amb & (d < n_h)
    base = np.zeros(n_h)
    np.add.at(base, d[sure], amp[sure])
    base_cnt = np.bincount(d[sure], minlength=n_h)[:n_h]
    idx = np.flatnonzero(amb)
    want = base.copy()
    if idx.size == 0:
        return want, 0
    g64 = np.asarray(got, np.float64)
    idx = idx[np.argsort(m[idx], kind="stable")]
    groups, cur = [], [int(idx[0])]
    for i in idx[1:]:
        if m[i] - m[cur[-1]] <= 1:
            cur.append(int(i))
        else:
            groups.append(cur)
            cur = [int(i)]
    groups.append(cur)
    for grp in groups:
        lo, hi = int(m[grp[0]]), min(int(m[grp[-1]]) + 2, n_h)
        amps = [amp[i] for i in grp]
        if len(grp) <= 12:
            best, best_s = None, None
            for choice in range(1 << len(grp)):
                taps = [int(m[i]) + ((choice >> k) & 1) for k, i in enumerate(grp)]
                sc = _group_score(taps, amps, g64, base, base_cnt, lo, hi, n_h)
                if best_s is None or sc < best_s:
                    best, best_s = taps, sc
        else:
            best = [int(d[i]) for i in grp]
            best_s = _group_score(best, amps, g64, base, base_cnt, lo, hi, n_h)
            moved = True
            while moved:
                moved = False
                for k in range(len(grp)):
                    for k2 in [None] + list(range(k + 1, min(k + 4, len(grp)))):
                        trial = list(best)
                        for q in (k, k2):
                            if q is not None:
                                trial[q] = 2 * int(m[grp[q]]) + 1 - trial[q]
                        sc = _group_score(trial, amps, g64, base, base_cnt, lo, hi, n_h)
                        if sc < best_s:
                            best, best_s, moved = trial, sc, True
        for p, a in zip(best, amps):
            if p < n_h:
                want[p] += a
    return want, int(idx.size)


def check_rir(got, want, what):
    assert got.shape == want.shape, what
    assert np.all(np.isfinite(got)), what
    np.testing.assert_array_equal(np.flatnonzero(got), np.flatnonzero(want), err_msg=what)
    if not want.any():
        return
    err = got.astype(np.float64) - want
    assert np.linalg.norm(err) <= REL_L2 * np.linalg.norm(want), what
    assert np.max(np.abs(err)) <= MAX_ABS * np.max(np.abs(want)), what


def _near_threshold(h, eta_db, rel=1e-5):
    """True if some tap's power sits within `rel` of the Eq. 7 threshold (a
    truncation decision that FP32 rounding of the taps may flip)."""
    p = np.asarray(h, np.float64) ** 2
    if p.size == 0 or p.max() == 0:
        return False
    p_th = p.max() * 10.0 ** (-eta_db / 10.0)
    return bool(np.any(np.abs(p - p_th) <= rel * p_th))


def _valid_cut(h, L, eta_db, rel=1e-5):
    """L is a reading of Eq. 7-9 for taps h known to a relative 1e-5: every tap
    from L on is below the threshold and tap L - 2 (the last kept crossing) is
    not, each within that tolerance; or L = N_h when the last crossing is one
    of the final two taps."""
    p = np.asarray(h, np.float64) ** 2
    if not math.isfinite(eta_db):
        return L == len(h)
    p_th = p.max() * 10.0 ** (-eta_db / 10.0)
    if not np.all(p[L:] < p_th * (1 + rel)):
        return False
    if L == len(h):
        return bool(np.any(p[max(L - 2, 0):] >= p_th * (1 - rel)))
    return L >= 2 and p[L - 2] >= p_th * (1 - rel)


