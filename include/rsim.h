/*
 * rsim: GPU room-simulator filter-and-mix (C ABI).
 *
 * Computes, for a batch of utterances, the far-field microphone signals of
 * the room simulator (Kim et al., "Efficient Implementation of the Room
 * Simulator for Training Deep Neural Network Acoustic Models"):
 *
 *   Eq. 7-9  hhat_ij = h_ij cut where its power falls eta dB below its peak
 *   Eq. 2    y_j[n]  = sum_i alpha_i (hhat_ij * x_i)[n],  n in [0, Ny)
 *
 * with Ny = Nx ("same" output, the default) or Ny = Nx + max_ij Nh_ij - 1
 * (the full convolution of the untruncated RIR lengths; samples past
 * Nx + L_max - 1 are zero), chosen per plan by output_mode.
 *
 * by overlap-add FFT filtering (Sec. 2.2, Eq. 6), and its adjoint (gradients
 * with respect to x_i, h_ij and alpha_i; gain mode 2 takes Eq. 2's general
 * alpha_ij, one gain per source and microphone).  The library also generates
 * image-method RIRs (Eq. 1, rsim_image_rirs) and computes the log-Mel features
 * the paper trains on (Sec. 3, rsim_plan_log_mel).  All arithmetic runs in CUDA
 * kernels on one GPU; the library has no CPU fallback.
 *
 * Packed layouts (all FP32, device memory unless stated otherwise):
 *   x    [sum_u I_u * Nx_u]            utterance, then source, then sample
 *   rir  [sum_u sum_{i,j} Nh_uij]      utterance, then source i, then mic j,
 *                                      then tap; RIR index r = rir0_u + i*J + j
 *   y    [sum_u J * Ny_u]              utterance, then mic, then sample
 *   per-source arrays (snr_db, gains)  [sum_u I_u], utterance then source
 *   per-RIR arrays (trunc_len, ...)    [sum_u I_u * J], RIR index order
 * Source 0 of every utterance is the target; sources 1.. are noise sources.
 *
 * Ownership: every buffer passed to a call belongs to the caller and must
 * stay valid until the work queued on the call's stream has finished.  The
 * plan owns its scratch memory (allocated in rsim_plan, freed in
 * rsim_plan_destroy) and must not be used by two streams at once.
 *
 * Errors: every call returns an rsim_status; rsim_last_error() gives a
 * message for the calling thread's last failure.  Argument errors are found
 * on the host before any work is queued.  Conditions only the device can see
 * (a truncated RIR longer than every allowed FFT size permits, a silent noise
 * source that must meet an SNR) are latched in the plan and reported by
 * rsim_plan_sync_status().
 */
#ifndef RSIM_H_
#define RSIM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsim_plan_s *rsim_plan_t;

typedef enum {
    RSIM_OK = 0,
    RSIM_E_INVALID = 1,      /* bad argument (shape, pointer, value) */
    RSIM_E_UNSUPPORTED = 2,  /* valid request outside what the kernels support */
    RSIM_E_NOMEM = 3,        /* device allocation failed */
    RSIM_E_CUDA = 4,         /* a CUDA runtime call failed */
    RSIM_E_DEVICE = 5,       /* error latched by a kernel (see rsim_last_error) */
    RSIM_E_STATE = 6         /* call out of order (backward before forward) */
} rsim_status;

/* Shapes and options of a plan (host memory, copied by rsim_plan). */
typedef struct {
    int32_t num_utts;              /* U >= 1 */
    int32_t num_mics;              /* J >= 1, shared by the batch */
    const int32_t *num_sources;    /* [U], 1 <= I_u <= 16 */
    const int64_t *num_samples;    /* [U], Nx_u >= 1 */
    const int32_t *rir_len;        /* [sum_u I_u J], Nh >= 1 (before the cut-off) */
    double eta_db;                 /* Eq. 7 threshold in dB, >= 0; +INFINITY keeps every tap */
    int32_t fft_sizes_mask;        /* bit m allows N = 2^m, m in [11, 14]; 0 = all of them */
    int32_t gain_mode;             /* 0: alpha from SNRs on the dry signals (computed,
                                         written to gains);
                                      1: alpha given by the caller in gains;
                                      2: one alpha_ij per (source, microphone), Eq. 2's
                                         general form, given by the caller in gains [R];
                                      3: alpha from SNRs on the reverberant signals at
                                         microphone snr_ref_mic (computed, written) */
    int64_t segment_len;           /* samples per forward work tile; 0 = default (the largest
                                      allowed N); raised to the largest allowed N */
    int64_t bwd_segment_len;       /* unused (kept for the layout): the backward of each FFT
                                      size is cut on the device into one contiguous run of
                                      blocks of equal cost per CTA of its launch */
    const float *fft_cost;         /* [32] host, relative cost of one real FFT of size 2^m
                                      used to pick N per utterance; NULL = N log2 N */
    int32_t disable_graphs;        /* 0: each call replays a CUDA graph of its launch sequence,
                                      captured on the first call with a given set of buffer
                                      pointers; 1: launch eagerly */
    int32_t output_mode;           /* 0: "same" output, Ny = Nx; 1: full output,
                                      Ny = Nx + (longest RIR of the utterance) - 1 */
    int32_t snr_ref_mic;           /* gain_mode 3: the microphone j (0 <= j < J) whose
                                      reverberant signal sets the SNRs; ignored otherwise */
    int32_t rooms;                 /* 1: the plan also serves rsim_filter_mix_rooms (RIRs made
                                      from room geometry on the device; reserves the kept taps,
                                      sum Nh floats); needs gain_mode 0, 1 or 2, every Nh at
                                      most 40960 and an RIR within the largest FFT size's
                                      reach (no partitioned convolution); 0: not */
    int32_t long_rirs;             /* with a cut-off (finite eta_db): 1 gives every utterance
                                      whose untruncated RIRs reach beyond one block of the
                                      largest allowed FFT size a partitioned path (see
                                      rsim_plan), taken on the device when its kept RIRs do
                                      too; 0: a kept RIR beyond that reach is reported by
                                      rsim_plan_sync_status (RSIM_E_UNSUPPORTED).  Without a
                                      cut-off those utterances always take the partitioned
                                      path, whatever this field says. */
    int32_t spectrum_cache;        /* 1: the forward keeps each block's source half spectrum
                                      X_ib, which the backward reads instead of transforming
                                      the block again: up to N = 8192 the same spectra, so
                                      the same results; at N = 16384 the two kernels
                                      transform with different thread shapes, so results
                                      differ from those without the cache by FP32 rounding
                                      only; the plan reserves at most 16 bytes per source
                                      sample (plus one block) for them; 0: no cache */
} rsim_plan_desc;

/* Creates a plan for the given shapes on CUDA device `device`.  Validates the
 * description, allocates scratch and uploads twiddle tables.  On success *out
 * holds a plan to be released with rsim_plan_destroy.
 *
 * One block of the largest allowed FFT size N reaches RIRs of 3N/4 + 1 taps
 * (hop >= N/4).  An utterance whose untruncated RIRs are longer (without a
 * cut-off, or with one and long_rirs = 1) also gets a partitioned path
 * (Sec. 2.2, Eq. 6, computed in pieces): source i delayed by p * N/2 samples is
 * filtered by taps [p N/2, (p+1) N/2) of its RIRs, for p < ceil(longest RIR of
 * the utterance / (N/2)), and the parts are summed -- the same Eq. 2.  The
 * planner on the device sends an utterance there when its kept RIRs do not fit
 * one block (always without a cut-off); the parts of a kept RIR are zero from
 * its kept length L on, so the result is the mix with the cut RIRs.  Every
 * output range and gain mode is served; at most 64 sources times parts per
 * utterance (RSIM_E_UNSUPPORTED otherwise).  Its scratch holds the delayed
 * copies of those utterances' sources over the output range.  With gain_mode 3
 * the plan also filters every source to the reference microphone (a second,
 * one-microphone plan inside this one).  A plan with a partitioned path cannot
 * be reshaped. */
rsim_status rsim_plan(const rsim_plan_desc *desc, int device, rsim_plan_t *out);

/* Forward filter-and-mix (Eq. 7-9 truncation, gains, Eq. 2 by overlap-add).
 *   stream            cudaStream_t to queue the work on (NULL = legacy default)
 *   x                 packed sources, read only
 *   rir               packed RIRs, read only
 *   snr_db            [sum I_u] SNR of each noise source in dB relative to the
 *                     utterance's target (dry-signal mean power over [0, Nx));
 *                     entry of the target ignored.  Used when gain_mode = 0
 *                     (P the dry signal's mean square) or 3 (P the mean square
 *                     over [0, Nx) of the source filtered by its cut RIR to
 *                     microphone snr_ref_mic); may be NULL otherwise.
 *   gains             [sum I_u] alpha_i: written when gain_mode = 0 (alpha_0 = 1,
 *                     alpha_i = sqrt(P_0 / P_i * 10^(-SNR_i/10))), read when 1;
 *                     gain_mode 2: [R] alpha_ij in RIR order, read (each is folded
 *                     into its RIR's spectrum; the cut-off uses the unscaled RIR)
 *   y                 packed output, overwritten
 *   trunc_len         [R] int32 kept lengths L (Eq. 9), or NULL
 *   energy_kept_frac  [R] sum_{n<L} h^2 / sum_n h^2, or NULL
 * The call is asynchronous.  The plan keeps the truncation lengths, the FFT
 * sizes and the RIR spectra for the next rsim_filter_mix_backward.  Unless
 * the plan disables graphs (or stage timing is on), the first call with a
 * given set of pointers captures the launch sequence into a CUDA graph and
 * every call replays it on `stream` (the plan keeps the graphs of the four
 * most recently used pointer sets, so alternating between double buffers
 * replays); the capture itself runs on a stream of the plan, so `stream` may
 * be the legacy default stream.  Calls on one plan must not overlap on the
 * GPU (they share the plan's scratch): queue them on one stream, or order
 * them with events. */
rsim_status rsim_filter_mix(rsim_plan_t plan, void *stream, const float *x, const float *rir,
                            const float *snr_db, float *gains, float *y, int32_t *trunc_len,
                            float *energy_kept_frac);

/* Adjoint of the last rsim_filter_mix on this plan (same x, rir and gains
 * buffers, unchanged).  With grad_y = dLoss/dy:
 *   grad_x     [like x]    alpha_i sum_j (hhat_ij correlated with grad_y_j)
 *   grad_rir   [like rir]  alpha_i (grad_y_j correlated with x_i) for taps < L,
 *                          0 for taps >= L (the cut-off is a fixed mask)
 *   grad_gains [sum I_u]   <grad_y_j, hhat_ij * x_i> summed over j; gains are
 *                          treated as inputs (no gradient flows to the SNRs)
 * With gain_mode 2, alpha_ij takes the place of alpha_i above, and grad_gains
 * is [R]: <grad_y_j, hhat_ij * x_i> per RIR (it reads the rir buffer the last
 * forward was given).
 * grad_y has the layout of y (Ny samples per mic, per the plan's output_mode).
 * grad_x may be NULL (not computed); grad_rir and grad_gains must be given.
 * Returns RSIM_E_STATE if no forward ran on the plan.  Asynchronous. */
rsim_status rsim_filter_mix_backward(rsim_plan_t plan, void *stream, const float *grad_y,
                                     const float *x, const float *gains, float *grad_x,
                                     float *grad_rir, float *grad_gains);

/* Waits for the plan's stream work and reports errors latched by kernels
 * (RSIM_E_UNSUPPORTED: no allowed FFT size N has N >= 4 (N - L_max + 1), with L_max the
 * longest truncated RIR of an utterance;
 * RSIM_E_INVALID: a noise source has zero power;
 * RSIM_E_DEVICE: a kernel's bounded wait (about half a second) for one of its own bulk
 * copies into shared memory ran out; the kernel stopped early and the outputs of that
 * call are invalid, the context stays usable).  Clears the latch.  For tests only, a plan
 * made while the environment variable RSIM_TEST_WITHHOLD_BULK_COPY=1 is set issues no
 * bulk copy, so that path can be exercised without any device fault. */
rsim_status rsim_plan_sync_status(rsim_plan_t plan, void *stream);

/* Copies the per-utterance plan chosen on the device by the last forward:
 * log2 of the FFT size, hop (N - L_max + 1), L_max and block count, each [U]
 * int32 host arrays (any may be NULL); for an utterance the planner sent to
 * its partitioned path, the size, hop and blocks of that filtering (L_max
 * stays the longest kept RIR).  Synchronises the stream. */
rsim_status rsim_plan_query(rsim_plan_t plan, void *stream, int32_t *log2_n, int32_t *hop,
                            int32_t *l_max, int32_t *num_blocks);

/* Stage timing.  When enabled, later calls record CUDA events on their
 * stream around each stage; rsim_plan_stage_times() synchronises the plan's
 * device, adds up the recorded durations (at most the last 64 calls) and
 * resets them.  Stages, in array order:
 *   0 truncation (Eq. 7-9)     1 source power and gains
 *   2 planner (N, queues, backward partition)       3 RIR spectra
 *   4 OLA forward              5 segment fix-up
 *   6 OLA backward             7 backward reduction
 * ms[8] receives milliseconds summed over calls, calls[8] the number of calls
 * summed (either may be NULL). */
#define RSIM_NUM_STAGES 8
rsim_status rsim_plan_set_timing(rsim_plan_t plan, int enable);
rsim_status rsim_plan_stage_times(rsim_plan_t plan, double *ms, int32_t *calls);

/* Bytes of device scratch owned by the plan. */
int64_t rsim_plan_scratch_bytes(rsim_plan_t plan);

/* Upper-bound plans: re-plans `plan` for another batch shape in place, without
 * new device memory, streams or events (a plan per shape class rather than
 * per batch: Sec. 1 draws fresh rooms and utterances every epoch, so a training
 * loop meets a new shape on every batch).  A plan made for the largest batch of a class serves every
 * batch whose scratch pieces each fit the class's: fewer or shorter
 * utterances, fewer sources, shorter RIRs.  Only num_utts, num_sources,
 * num_samples, rir_len and fft_cost may differ from the plan's description;
 * plans with partitioned convolution or gain_mode 3 are not reshaped.  Waits
 * for the device to finish the plan's earlier work, then uploads the new
 * tables; the captured graphs of the old shape are dropped and a backward
 * needs a forward of the new shape first.
 * Errors: RSIM_E_INVALID (a fixed field differs), RSIM_E_UNSUPPORTED (the
 * batch does not fit the class, or needs partitioned convolution: make a new
 * plan); on error the plan keeps its old shape. */
rsim_status rsim_plan_reshape(rsim_plan_t plan, const rsim_plan_desc *desc);

/* Releases the plan and its device memory (NULL is ignored).  The caller must
 * make sure no queued work still uses it. */
void rsim_plan_destroy(rsim_plan_t plan);

/* Allocation-free per-source gains.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they need the gains -- code running under a memory manager that owns every
 * device allocation (a framework's caching allocator, a real-time audio
 * engine that reserves its memory at start-up) or code where an allocation
 * would stall the device at the wrong moment.  rsim_plan allocates, so such
 * callers cannot make a plan.
 *
 * Computes, for a batch laid out as for rsim_filter_mix, the gains
 * rsim_filter_mix writes with gain_mode = 0: alpha_0 = 1 and
 * alpha_i = sqrt(P_0 / P_i * 10^(-SNR_i/10)), P the mean square of the dry
 * source over [0, Nx); a noise source with P_i = 0 gets NaN.
 *   stream       cudaStream_t (NULL = legacy default stream)
 *   num_utts     U >= 1
 *   num_sources  [U] host, 1..16 sources per utterance
 *   num_samples  [U] host, Nx >= 1
 *   x            packed sources, device, read only
 *   snr_db       [sum I_u] device (entry of each target ignored)
 *   gains        [sum I_u] device, written
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch
 * is one fixed 2 MiB device array inside the library, present on every GPU
 * that loads the library until the process exits; a batch needing more
 * (about 8 bytes per source per 32768 samples of the longest utterance plus
 * 28 bytes per source and utterance) is rejected with RSIM_E_UNSUPPORTED and
 * a message.  Nothing in the scratch has to start at zero: each call writes
 * every entry it reads.  All calls share that one array, so calls whose work
 * overlaps on the GPU race; queue them on one stream or wait between them.
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture, and do not call this entry point again on a
 * device after cudaDeviceReset has been called for it (the kept address would
 * be stale).  num_sources and num_samples are copied to the device on
 * `stream` with cudaMemcpyAsync: from pageable host memory that copy is
 * finished when the call returns (it may wait for earlier work on the
 * stream); from pinned host memory it is not, and the arrays must stay
 * unchanged until the stream has reached the call.  Asynchronous otherwise. */
rsim_status rsim_source_gains_noalloc(void *stream, int32_t num_utts, const int32_t *num_sources,
                                      const int64_t *num_samples, const float *x, const float *snr_db,
                                      float *gains);

/* ---- log-Mel front end (Sec. 3) ---------------------------------------------
 *
 * The features the paper trains on, from one microphone of the mixed output:
 * frames of 512 samples (32 ms at 16 kHz) every `hop` samples (160: 10 ms),
 * frame t covering [t hop, t hop + 512) of the utterance's N_y samples with no
 * padding (T = (N_y - 512) / hop + 1 frames, none if N_y < 512); a periodic
 * Hann window 1/2 - 1/2 cos(2 pi n / 512); the power spectrum |X[k]|^2,
 * k = 0 .. 256; n_mels triangular filters whose n_mels + 2 edges are equally
 * spaced on the HTK Mel scale m(f) = 2595 log10(1 + f / 700) from f_lo to
 * f_hi (filter j rises from edge j to edge j+1 and falls to edge j+2, peak 1);
 * v = ln(E + log_floor) per filter; then `stack` consecutive frames side by
 * side per row, one row every `stride` frames (the paper: 128 filters over
 * 125-7500 Hz, 4 frames stacked, every third kept).  Row r of an utterance
 * holds frames stride r .. stride r + stack - 1 (frame-major, n_mels values
 * each), for every r whose frames all exist: R = (T - stack) / stride + 1
 * rows (none if T < stack).  feats is [sum_u R_u, stack * n_mels] FP32,
 * utterances in order.  The filter edges are computed in FP64 on the host and
 * rounded once; everything else runs in FP32 on the device.
 */
typedef struct {
    int32_t channel;    /* microphone j, 0 <= j < J */
    int32_t hop;        /* samples between frames, >= 1 */
    float fs;           /* sampling rate in Hz, > 0 */
    int32_t n_mels;     /* filters, 1 .. 128 */
    float f_lo, f_hi;   /* Hz, 0 <= f_lo < f_hi <= fs / 2 */
    float log_floor;    /* added to each filter energy before the log, > 0 */
    int32_t stack;      /* frames per row, >= 1 */
    int32_t stride;     /* frames between rows, >= 1 */
} rsim_mel_desc;

/* Rows per utterance (rows_per_utt [U] host, may be NULL) and their total
 * (may be NULL) of the features rsim_plan_log_mel writes for this plan's
 * output lengths.  Host only; RSIM_E_INVALID for a bad description. */
rsim_status rsim_plan_log_mel_rows(rsim_plan_t plan, const rsim_mel_desc *desc, int64_t *rows_per_utt,
                                   int64_t *total_rows);

/* Writes the features of desc->channel of y (laid out as rsim_filter_mix writes
 * it for this plan, device, read only) into feats (device, caller-owned, the
 * total rows times stack * n_mels floats; may be NULL when there are no rows).
 * Uses the plan's scratch for the row
 * offsets, so calls on one plan must not overlap.  RSIM_E_UNSUPPORTED for more
 * than 65535 utterances.  Asynchronous; no allocation. */
rsim_status rsim_plan_log_mel(rsim_plan_t plan, void *stream, const float *y, const rsim_mel_desc *desc,
                              float *feats);

/* ---- image-method room impulse responses (Eq. 1, Sec. 2) -------------------
 *
 * One RIR per (source, microphone) pair of a cuboid room by the image method:
 *     h[n] = sum_v r^g_v / d_v * delta[n - ceil(d_v fs / c0)],   0 <= n < n_h,
 * summed over the images of the source in the (2K+1)^3 virtual rooms (a, b, c),
 * |a|, |b|, |c| <= K, that mirroring the room across its walls produces (the
 * paper uses K = 8: 17^3 = 4913 rooms, fs = 16 kHz, c0 = 343 m/s).  The room
 * is the box [0, Lx] x [0, Ly] x [0, Lz]; along one axis virtual room a spans
 * [a L, (a+1) L] and holds the image a L + s (a even) or (a+1) L - s (a odd),
 * reached after |a| reflections, so g_v = |a| + |b| + |c|.  d_v is the image's
 * distance to the microphone and r the reflection coefficient of every wall.
 *
 * The delay is an integer decision made in FP32, as ceil(d * rate) with
 * rate = fs / c0: image coordinate, offset to the microphone, squares, their
 * sum (x + y) + z, square root, the rate and the product are each one
 * correctly rounded FP32 operation, so the delay of every image is
 * reproducible bit for bit.  Amplitudes are FP32 (r^|a| r^|b| r^|c|, each by
 * repeated squaring, times an approximate 1/d) and summed in shared memory in
 * no fixed order: taps where images collide can differ in the last bits from
 * call to call.  An image whose delay is n_h or later is dropped.
 *
 * The output has the packed layout rsim_filter_mix reads: RIR r occupies
 * rir[rir_off[r] .. rir_off[r+1]), so rsim_plan_desc.rir_len[r] must be
 * rir_off[r+1] - rir_off[r] for the generated RIRs to feed the mix directly.
 */
typedef struct {
    float room[3];   /* Lx, Ly, Lz in metres, each > 0 and finite */
    float src[3];    /* source position, strictly inside the room */
    float mic[3];    /* microphone position, strictly inside the room, not at the source */
    float refl;      /* wall reflection coefficient r, 0 <= r < 1 (r = 0: direct path only) */
} rsim_image_geom;

/*   stream     cudaStream_t (NULL = legacy default stream)
 *   num_rirs   R >= 0 (0: nothing but the status reset)
 *   geom       [R] device, read only
 *   rir_off    [R+1] device, read only: nondecreasing offsets into rir; every
 *              length rir_off[r+1] - rir_off[r] at most 2^24 taps
 *   max_len    host: the longest length, in [0, 2^24]; it sizes the grid only
 *              (a longer RIR is still written whole)
 *   order      K in [0, 32]
 *   fs, c0     sampling rate (Hz) and speed of sound (m/s), finite and > 0
 *   rir        device, written on [rir_off[0], rir_off[R]) (caller-owned)
 *   status     device int32 or NULL; set to 0, then bit 1 is set if some
 *              geometry is invalid (its RIR is written as zeros) and bit 2 if
 *              some length is negative or above 2^24 (that RIR is not written)
 * Returns RSIM_E_INVALID for a bad host argument, RSIM_E_CUDA if the launch
 * fails; asynchronous otherwise.  No allocation; safe to capture in a graph. */
rsim_status rsim_image_rirs(void *stream, int32_t num_rirs, const rsim_image_geom *geom,
                            const int64_t *rir_off, int64_t max_len, int32_t order, float fs, float c0,
                            float *rir, int32_t *status);

/* ---- RIRs generated where they are consumed (Eq. 1 into Eq. 7-9 and Eq. 2) --
 *
 * The forward of rsim_filter_mix with the RIRs made on the device from room
 * geometry instead of read from the caller: one kernel per call lands every
 * image of each RIR (Eq. 1, as rsim_image_rirs computes it, the plan's
 * rir_len[r] taps) in on-chip shared memory, takes the Eq. 7-9 cut-off there
 * with the same decision as rsim_filter_mix, and writes only the kept taps
 * [0, L) to the plan's scratch, from which the RIR spectra are taken; the full
 * RIRs never pass through device memory unless rir_out asks for them.  The plan
 * must have been made with rooms = 1.
 *   geom       [R] device, one room geometry per RIR in RIR index order (the
 *              room, source and microphone of RIR r = rir0_u + i J + j)
 *   order      K in [0, 32]: (2K + 1)^3 virtual rooms
 *   fs, c0     sampling rate (Hz) and speed of sound (m/s), finite and > 0
 *   rir_out    [sum Nh] device or NULL: if given, receives every tap of the
 *              generated RIRs (as rsim_image_rirs would write them)
 *   the other arguments as rsim_filter_mix.
 * A geometry that is invalid or puts an image at the microphone gives that
 * RIR all zeros (L = 1) and is reported as RSIM_E_INVALID by
 * rsim_plan_sync_status.  A later rsim_filter_mix_backward on the plan is the
 * adjoint of this forward, with dh over the generated RIRs' taps.
 * Asynchronous; graphs as for rsim_filter_mix. */
rsim_status rsim_filter_mix_rooms(rsim_plan_t plan, void *stream, const float *x, const rsim_image_geom *geom,
                                  int32_t order, float fs, float c0, const float *snr_db, float *gains,
                                  float *y, int32_t *trunc_len, float *energy_kept_frac, float *rir_out);

/* Message describing the calling thread's last error ("" if none). */
const char *rsim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RSIM_H_ */
