"""Seeded synthetic inputs shaped like the room simulator's workloads.

This module only *draws* inputs: speech stand-ins, noise sources, room
impulse responses, SNRs and the batch bookkeeping (offsets of the packed
arrays).  It holds none of the method's arithmetic (no truncation, no gains,
no filtering), so both the CUDA path and the FP64 oracle can be fed from it.

Workload shapes follow the paper's statistics:
  * utterances are 16 kHz, mean length 7.31 s (Sec. 2.2);
  * J = 2 microphones 7.1 cm apart (Sec. 3);
  * 0-3 noise sources besides the target, mean I = 2.55 (Sec. 2.1);
  * reverberation times around 0.48 s (Table 4).
The paper's data sets are not available; these generators stand in for them.

Recipe (all draws from numpy PCG64):
  * speech stand-in: AR(2) Gaussian process with poles 0.9*exp(+-0.3i)
    (x[n] = 1.719606 x[n-1] - 0.81 x[n-2] + e[n]), 1000-sample burn-in,
    scaled to peak 0.5;
  * noise source: white Gaussian or AR(1) with coefficient 0.95 (50/50),
    scaled to peak 0.5;
  * RIR: N(0, 0.1^2) noise times exp(-6.91 n / (RT60 fs)) for
    n < ceil(RT60 fs), plus a direct impulse 1/r at d0 = round(fs r / 343),
    where r is the source-to-microphone distance;
  * SNR: uniform in [0, 30] dB per noise source.

Rooms for the image-method RIRs (`room_geometry`):
  * one cuboid room per utterance, Lx ~ U(3, 10), Ly ~ U(3, 8), Lz ~ U(2.5, 5) m;
  * RT60 ~ U(0.1, 0.9) s; every wall's reflection coefficient follows from
    Sabine's formula, r = sqrt(1 - a) with a = 0.161 V / (S RT60) clipped to
    [0.01, 0.99] (V the volume, S the wall area);
  * the microphone array (the same geometry as above, in the horizontal
    plane, turned by a random azimuth) is centred at a uniform point at least
    0.8 m from the side walls, 0.8-1.8 m high; each source sits at a
    distance U(1, 3) m and azimuth U(0, 2 pi) from the centre, up to 0.5 m
    above or below it, moved inside the room (0.3 m from every wall) if it
    falls outside;
  * every RIR of an utterance has ceil(RT60 fs) taps, as above.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FS = 16000          # sampling rate used by the room simulator (Sec. 2.1)
C0 = 343.0          # speed of sound in m/s (Sec. 2.1)
SEED_BASE = 171203439


@dataclasses.dataclass
class Batch:
    """A batch of utterances in the packed layout the library consumes.

    x      float32 [sum_u I_u * Nx_u]          source-major within an utterance
    rir    float32 [sum_u sum_{i,j} Nh_uij]    order (u, i, j, tap)
    snr_db float32 [sum_u I_u]                 entry of the target (i = 0) unused
    y      float32 [sum_u J * Nx_u]            mic-major within an utterance
    """
    num_mics: int
    num_sources: np.ndarray     # int32 [U]
    num_samples: np.ndarray     # int64 [U]
    rir_len: np.ndarray         # int32 [sum_u I_u * J]
    x: np.ndarray               # float32
    rir: np.ndarray             # float32
    snr_db: np.ndarray          # float32

    @property
    def num_utts(self) -> int:
        return int(self.num_sources.shape[0])

    @property
    def num_rirs(self) -> int:
        return int(self.rir_len.shape[0])

    # ---- offsets of the packed arrays (pure bookkeeping) -------------------
    def src_index(self) -> np.ndarray:
        """First source index of each utterance, [U+1]."""
        return np.concatenate([[0], np.cumsum(self.num_sources.astype(np.int64))])

    def x_offsets(self) -> np.ndarray:
        """Offset of source (u, i) in x, flattened in source order, [sum I + 1]."""
        lens = np.repeat(self.num_samples, self.num_sources)
        return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)

    def rir_offsets(self) -> np.ndarray:
        """Offset of RIR r in rir, [R + 1]."""
        return np.concatenate([[0], np.cumsum(self.rir_len.astype(np.int64))])

    def rir_index(self) -> np.ndarray:
        """First RIR index of each utterance, [U+1]."""
        per = self.num_sources.astype(np.int64) * self.num_mics
        return np.concatenate([[0], np.cumsum(per)])

    def y_offsets(self) -> np.ndarray:
        """Offset of utterance u in y, [U+1]."""
        per = self.num_samples * self.num_mics
        return np.concatenate([[0], np.cumsum(per)]).astype(np.int64)

    @property
    def y_size(self) -> int:
        return int(np.sum(self.num_samples) * self.num_mics)

    def audio_seconds(self) -> float:
        """Target-utterance seconds in the batch (not multiplied by I or J)."""
        return float(np.sum(self.num_samples)) / FS

    def excerpt(self, n_max: int) -> "Batch":
        """The same batch with every utterance cut to its first min(Nx, n_max)
        samples (all its sources alike; RIRs and SNRs unchanged)."""
        xo, si = self.x_offsets(), self.src_index()
        n_new = np.minimum(self.num_samples, int(n_max)).astype(np.int64)
        xs = []
        for u in range(self.num_utts):
            for s in range(si[u], si[u + 1]):
                xs.append(self.x[xo[s]:xo[s] + n_new[u]])
        return dataclasses.replace(self, num_samples=n_new, x=np.concatenate(xs).astype(np.float32))

    def subset(self, utts) -> "Batch":
        """A batch made of the given utterance indices (in that order)."""
        utts = list(utts)
        si, xo, ri, ro = self.src_index(), self.x_offsets(), self.rir_index(), self.rir_offsets()
        xs, rs, lens, snrs = [], [], [], []
        for u in utts:
            s0, s1 = si[u], si[u + 1]
            xs.append(self.x[xo[s0]:xo[s1]])
            snrs.append(self.snr_db[s0:s1])
            r0, r1 = ri[u], ri[u + 1]
            rs.append(self.rir[ro[r0]:ro[r1]])
            lens.append(self.rir_len[r0:r1])
        return Batch(self.num_mics,
                     self.num_sources[utts].copy(), self.num_samples[utts].copy(),
                     np.concatenate(lens).astype(np.int32),
                     np.concatenate(xs).astype(np.float32),
                     np.concatenate(rs).astype(np.float32),
                     np.concatenate(snrs).astype(np.float32))


# ---------------------------------------------------------------------------
# signal generators
# ---------------------------------------------------------------------------
def _lfilter(b, a, e):
    from scipy.signal import lfilter
    return lfilter(b, a, e)


def _peak_normalise(s: np.ndarray, peak: float = 0.5) -> np.ndarray:
    m = float(np.max(np.abs(s))) if s.size else 0.0
    if m > 0:
        s = s * (peak / m)
    return s


def speech_like(rng: np.random.Generator, n: int) -> np.ndarray:
    """AR(2) Gaussian process with poles 0.9 exp(+-0.3i), peak 0.5."""
    burn = 1000
    e = rng.standard_normal(n + burn)
    a1 = 2.0 * 0.9 * math.cos(0.3)   # 1.719606...
    s = _lfilter([1.0], [1.0, -a1, 0.81], e)[burn:]
    return _peak_normalise(s).astype(np.float32)


def noise_like(rng: np.random.Generator, n: int) -> np.ndarray:
    """White Gaussian or AR(1) (coefficient 0.95) noise, 50/50, peak 0.5."""
    if rng.random() < 0.5:
        s = rng.standard_normal(n)
    else:
        burn = 1000
        e = rng.standard_normal(n + burn)
        s = _lfilter([1.0], [1.0, -0.95], e)[burn:]
    return _peak_normalise(s).astype(np.float32)


def exp_decay_rir(rng: np.random.Generator, rt60: float, r: float,
                  n_taps: int | None = None) -> np.ndarray:
    """Exponential-decay RIR: decaying Gaussian tail plus a direct impulse 1/r."""
    if n_taps is None:
        n_taps = int(math.ceil(rt60 * FS))
    n = np.arange(n_taps)
    h = rng.normal(0.0, 0.1, n_taps) * np.exp(-6.91 * n / (rt60 * FS))
    d0 = int(round(FS * r / C0))
    if d0 < n_taps:
        h[d0] += 1.0 / r
    return h.astype(np.float32)


def linear_pair_array(spacing: float = 0.071) -> np.ndarray:
    """Two microphones on the x axis, `spacing` metres apart, centred at 0."""
    return np.array([[-spacing / 2, 0.0], [spacing / 2, 0.0]])


def circular_array(n_mics: int, radius: float) -> np.ndarray:
    ang = 2 * np.pi * np.arange(n_mics) / n_mics
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)


# ---------------------------------------------------------------------------
# batch generator
# ---------------------------------------------------------------------------
def make_batch(seed: int, lengths, n_sources, mics: np.ndarray, rt60_range,
               n_taps: int | None = None, snr_range=(0.0, 30.0),
               dist_range=(1.0, 3.0)) -> Batch:
    """Draws a batch.  `lengths` and `n_sources` are per-utterance sequences."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = np.asarray(lengths, dtype=np.int64)
    n_sources = np.asarray(n_sources, dtype=np.int32)
    J = int(mics.shape[0])
    xs, rirs, rlen, snrs = [], [], [], []
    for u in range(lengths.shape[0]):
        nx = int(lengths[u])
        I = int(n_sources[u])
        rt60 = float(rng.uniform(*rt60_range))
        for i in range(I):
            xs.append(speech_like(rng, nx) if i == 0 else noise_like(rng, nx))
            snrs.append(0.0 if i == 0 else float(rng.uniform(*snr_range)))
            r = float(rng.uniform(*dist_range))
            phi = float(rng.uniform(0.0, 2 * np.pi))
            src = np.array([r * math.cos(phi), r * math.sin(phi)])
            for j in range(J):
                rj = float(np.linalg.norm(src - mics[j]))
                h = exp_decay_rir(rng, rt60, rj, n_taps)
                rirs.append(h)
                rlen.append(h.shape[0])
    return Batch(J, n_sources, lengths,
                 np.asarray(rlen, dtype=np.int32),
                 np.concatenate(xs).astype(np.float32) if xs else np.zeros(0, np.float32),
                 np.concatenate(rirs).astype(np.float32),
                 np.asarray(snrs, dtype=np.float32))


def trim_rirs(batch: Batch, seed: int, min_frac: float = 0.3) -> Batch:
    """Cuts every RIR to a seeded length in [min_frac * Nh, Nh], so the RIRs of
    one utterance differ in length (the longest sets the full output length)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ro = batch.rir_offsets()
    keep = [max(1, int(rng.integers(int(math.ceil(min_frac * n)), n + 1))) for n in batch.rir_len]
    rir = np.concatenate([batch.rir[ro[r]:ro[r] + keep[r]] for r in range(batch.num_rirs)])
    return dataclasses.replace(batch, rir_len=np.asarray(keep, dtype=np.int32), rir=rir.astype(np.float32))


def output_lengths(batch: Batch, output_mode: int = 0) -> np.ndarray:
    """Samples per microphone of each utterance's output: Nx for the "same"
    output (mode 0), Nx + max Nh - 1 over the utterance's RIRs for the full one."""
    if not output_mode:
        return batch.num_samples.astype(np.int64).copy()
    ri = batch.rir_index()
    return np.array([int(batch.num_samples[u]) + int(batch.rir_len[ri[u]:ri[u + 1]].max()) - 1
                     for u in range(batch.num_utts)], dtype=np.int64)


def grad_like(seed: int, n: int, scale: float = 0.1) -> np.ndarray:
    """A seeded FP32 vector (an upstream gradient or a regression target)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, scale, n).astype(np.float32)


def room_geometry(seed: int, num_sources, mics: np.ndarray, rt60_range=(0.1, 0.9),
                  dist_range=(1.0, 3.0)):
    """Rooms, positions and wall reflection for the image-method RIRs of a batch
    shaped by `num_sources` (one room per utterance) and the array `mics`
    ([J, 2] offsets in metres).  Returns (geom float32 [R, 10] with rows
    (room, source, microphone, r) in the batch's (u, i, j) RIR order,
    rir_len int32 [R], rt60 [U])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    num_sources = np.asarray(num_sources, dtype=np.int64)
    J = int(mics.shape[0])
    rows, lens, rt60s = [], [], []
    margin = 0.3
    for u in range(num_sources.shape[0]):
        room = np.array([rng.uniform(3.0, 10.0), rng.uniform(3.0, 8.0), rng.uniform(2.5, 5.0)])
        rt60 = float(rng.uniform(*rt60_range))
        vol = float(np.prod(room))
        area = 2.0 * (room[0] * room[1] + room[0] * room[2] + room[1] * room[2])
        absorb = min(max(0.161 * vol / (area * rt60), 0.01), 0.99)
        refl = math.sqrt(1.0 - absorb)
        centre = np.array([rng.uniform(0.8, room[0] - 0.8), rng.uniform(0.8, room[1] - 0.8),
                           min(rng.uniform(0.8, 1.8), room[2] - margin)])
        turn = float(rng.uniform(0.0, 2 * np.pi))
        rot = np.array([[math.cos(turn), -math.sin(turn)], [math.sin(turn), math.cos(turn)]])
        mic_pos = [centre + np.append(rot @ mics[j], 0.0) for j in range(J)]
        n_h = int(math.ceil(rt60 * FS))
        for _ in range(int(num_sources[u])):
            dist = float(rng.uniform(*dist_range))
            phi = float(rng.uniform(0.0, 2 * np.pi))
            src = centre + np.array([dist * math.cos(phi), dist * math.sin(phi), rng.uniform(-0.5, 0.5)])
            src = np.clip(src, margin, room - margin)
            for j in range(J):
                rows.append(np.concatenate([room, src, mic_pos[j], [refl]]))
                lens.append(n_h)
        rt60s.append(rt60)
    return (np.asarray(rows, dtype=np.float32).reshape(-1, 10), np.asarray(lens, dtype=np.int32),
            np.asarray(rt60s))


# ---------------------------------------------------------------------------
# the five workloads (sizes as stated for the room-simulator benchmarks)
# ---------------------------------------------------------------------------
def config_tiny(seed: int = SEED_BASE + 0) -> Batch:
    """1 utterance of 16000 samples, 1 source, 1 mic, one 4800-tap RIR (RT60 0.3 s)."""
    return make_batch(seed, [16000], [1], np.zeros((1, 2)), (0.3, 0.3), n_taps=4800)


def config_home(seed: int = SEED_BASE + 1, n_utts: int = 256) -> Batch:
    """Google-Home-like mix: lengths U(2,15) s, 1 target + 0-3 noises, 2 mics 7.1 cm."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    lengths = (rng.uniform(2.0, 15.0, n_utts) * FS).astype(np.int64)
    n_src = 1 + rng.integers(0, 4, n_utts)
    return make_batch(seed, lengths, n_src, linear_pair_array(), (0.1, 0.9))


def config_diff(seed: int = SEED_BASE + 2, n_utts: int = 64) -> Batch:
    """The Home recipe at 64 utterances (differentiable mix)."""
    return config_home(seed, n_utts)


def config_fd_subcase(seed: int = SEED_BASE + 2) -> Batch:
    """2 utterances x 2000 samples, 256-tap RIRs (finite-difference sub-case)."""
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    n_src = 1 + rng.integers(0, 4, 2)
    return make_batch(seed, [2000, 2000], n_src, linear_pair_array(), (0.1, 0.3), n_taps=256)


def config_long(seed: int = SEED_BASE + 3, n_utts: int = 32) -> Batch:
    """32 x 30 s, 4 sources, 8-mic circle of radius 5 cm, RT60 U(0.8, 1.2)."""
    return make_batch(seed, [30 * FS] * n_utts, [4] * n_utts,
                      circular_array(8, 0.05), (0.8, 1.2))


def config_home_rooms(seed: int = SEED_BASE + 5, n_utts: int = 256):
    """The Home mix with image-method rooms in place of the drawn RIRs: returns
    (batch, geom), the batch's rir zero-filled (to be generated from geom)."""
    b = config_home(seed, n_utts)
    geom, rir_len, _ = room_geometry(seed + 3000, b.num_sources, linear_pair_array())
    return dataclasses.replace(b, rir_len=rir_len, rir=np.zeros(int(rir_len.astype(np.int64).sum()),
                                                                  np.float32)), geom


def config_stream(seed: int = SEED_BASE + 4, n_utts: int = 4096) -> Batch:
    """4096 utterances, log-uniform 0.5-20 s, 1-4 sources, 2 mics."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    lengths = (np.exp(rng.uniform(math.log(0.5), math.log(20.0), n_utts)) * FS).astype(np.int64)
    n_src = 1 + rng.integers(0, 4, n_utts)
    return make_batch(seed, lengths, n_src, linear_pair_array(), (0.1, 0.9))
