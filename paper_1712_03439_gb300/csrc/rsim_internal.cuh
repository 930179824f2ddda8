// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsim.h"

namespace rsim {

// Supported overlap-add FFT sizes N = 2^m, m in [kMinLog, kMaxLog]; the
// complex transform size is M = N/2.
constexpr int kMinLog = 11;
constexpr int kMaxLog = 14;
constexpr int kNumBuckets = kMaxLog - kMinLog + 1;
constexpr int kMaxSources = 16;      // sources per utterance (the public limit; the dalpha
                                     // partials are strided by it)
constexpr int kMaxPartSources = 64;  // virtual sources (source x part) per utterance of a
                                     // partitioned plan
constexpr int kJG = 2;               // microphones per group inside a tile
constexpr int kPowerChunk = 32768;   // samples per partial-power CTA

// device error word bits (latched, read by rsim_plan_sync_status)
enum : int32_t {
    kErrNoFftSize = 1,     // a truncated RIR longer than 3N/4+1 for every allowed N
    kErrZeroPower = 2,     // a noise source with zero power but an SNR to meet
    kErrWaitTimeout = 4,   // a kernel gave up waiting for a bulk copy (bounded wait)
    kErrBadGeometry = 8,   // a room geometry is invalid or puts an image at the microphone
    kErrBounds = 16,       // bounds-checked build: a store fell outside its buffer (skipped)
};

// list kinds inside the work queues
enum : int { kListFwd = 0, kListBwd = 1, kListSpec = 2, kNumLists = 3 };

// Batch description and per-call state on the device.  Utterance u has
// n_src[u] sources (source 0 is the target) and J microphones.  The forward
// cuts it into ceil(n_x / seg_len) segments, one tile each; the backward of
// each FFT size is cut into one contiguous chunk per CTA (for_each_piece).
struct DevBatch {
    int32_t U, J, S, R, IMAX;
    int32_t NSEG;            // total segments
    int32_t MMAX;            // largest allowed N/2 (spectrum cache stride)
    int32_t mask;            // allowed log2 N bitmask
    int64_t seg_len;         // samples per segment (>= largest allowed N)
    int32_t gain_mode;
    const int32_t* n_src;    // [U]
    const int64_t* n_x;      // [U] input samples
    const int64_t* n_y;      // [U] output samples per mic (Nx, or the full length)
    const int32_t* src0;     // [U+1] first source of utterance
    const int32_t* rir0;     // [U+1] first RIR of utterance
    const int32_t* seg0;     // [U+1] first segment of utterance
    const int32_t* seg_utt;  // [NSEG] utterance of segment
    const int64_t* xoff;     // [S+1] offset of source s in x
    const int64_t* yoff;     // [U+1] offset of utterance u in y
    const int64_t* roff;     // [R+1] offset of RIR r in rir
    const int32_t* rir_len;  // [R]
    const int32_t* src_utt;  // [S] utterance of source s
    const int32_t* rir_utt;  // [R] utterance of RIR r
    // backward partition (written by the planner; see for_each_piece below)
    int32_t PMAX;            // most CTAs of one FFT size's backward launch
    int32_t NPIECE;          // capacity of the piece arrays (S + sum of the launches' CTAs)
    int32_t bgrid[4];        // CTAs of each FFT size's backward launch
    int32_t* sord;           // [4][S] streams of each size in batch order (first source of the group)
    int64_t* spre;           // [4][S + 1] cost of the size's streams before each one (transforms)
    int32_t* nstream;        // [4] streams of each size
    int32_t* cta_sp;         // [4][PMAX + 1] first stream position of each CTA's chunk
    int32_t* cta_b;          // [4][PMAX + 1] first block in that stream
    int32_t* cta_p;          // [4][PMAX + 1] first piece of each chunk
    int64_t* piece_dh;       // [NPIECE] offset of each piece's RIR-gradient partials
    int64_t* lpre;           // [R + 1] kept taps of the RIRs before each one (the partials of a
                             // piece hold its stream's kept taps, RIR after RIR)
    int32_t* s_first;        // [S] first piece of the stream that starts at source s
    int32_t* s_last;         // [S] last piece of that stream
    const float* tuning;     // [32] cost per real FFT of size 2^m (any unit)
    // written on the device during a call
    int32_t* L;              // [R] kept RIR length (Eq. 9)
    int32_t* logN;           // [U] chosen log2 N (0 = none fits)
    int32_t* hop;            // [U]
    int32_t* Lmax;           // [U]
    int32_t* nblk;           // [U]
    double* pow_part;        // [S * CH] partial sums of x^2
    int32_t CH;              // power chunks per source (max)
    int32_t* err;            // [1] latched error bits
    int32_t test_withhold;   // test hook: the bulk copies are not issued, so the kernels'
                             // bounded waits run out (set from RSIM_TEST_WITHHOLD_BULK_COPY)
    int64_t NDHP;            // floats of the RIR-gradient partials (the planner fits the pieces in)
    // utterances whose RIRs may reach beyond one block of the largest size (partitioned path)
    const int64_t* defer_idx;   // [U] index of utterance u in the partitioned plan, -1 if it has
                                // none (NULL: no utterance has one)
    uint8_t* defer;             // [utterances of that plan] 1: the planner sent the utterance there
    const uint8_t* active;      // in the partitioned plan: [U] 0 = the outer planner kept the
                                // utterance (no work here); NULL: every utterance is active
    // source half spectra of every block, written by the forward for the backward (N <= 8192)
    float4* xspec;              // NULL: no cache.  Block b of source s: M/2 bin pairs from
                                // (char*)xspec + xspec_off[s] + b * M/2 * 16 bytes, pair k
                                // = (X[k], X[M - k]) (k = 0: (X[0], X[M]) packed, X[M/2])
    const int64_t* xspec_off;   // [S + 1] byte offset of each source's slots
    int64_t xspec_bytes;
};

struct Queues {
    int32_t* list;     // [kNumLists][kNumBuckets][cap]
    int32_t* count;    // [kNumLists][kNumBuckets]
    int32_t* next;     // [kNumLists][kNumBuckets] atomic cursors
    int32_t cap;       // capacity per (list, bucket)
    __host__ __device__ int32_t* lst(int kind, int b) const { return list + ((int64_t)kind * kNumBuckets + b) * cap; }
    __host__ __device__ int idx(int kind, int b) const { return kind * kNumBuckets + b; }
};

// The backward work of one FFT size is a sequence of streams -- (utterance, group
// of up to bwd_src_group(log2 N) of its sources), in batch order, each the
// utterance's nblk blocks long -- and each block of a stream costs
// kCostMic J + kCostSrc groups(J) I_g (I_g sources in the group), plus the
// stream's flush at its end.  The planner cuts the sequence at block boundaries
// into one chunk per CTA of the launch, of equal cost; a chunk is a list of pieces, the parts of the streams it covers
// (piece p: stream s, blocks [b0, b1)).  Pieces are numbered in sequence
// order, so a stream's pieces are consecutive (s_first[s] .. s_last[s]).
// Calls f(p, s, u, i0, b0, b1) for every piece of CTA k of size bucket b, in
// order (s = first source of the group, i0 = its index in the utterance).
template <typename F>
__device__ __forceinline__ void for_each_piece(const DevBatch& B, int b, int k, F f) {
    const int32_t* sp = B.cta_sp + (int64_t)b * (B.PMAX + 1);
    const int32_t* sb = B.cta_b + (int64_t)b * (B.PMAX + 1);
    const int pos0 = sp[k], blk0 = sb[k], pos1 = sp[k + 1], blk1 = sb[k + 1];
    int p = B.cta_p[(int64_t)b * (B.PMAX + 1) + k];
    for (int pos = pos0; pos <= pos1; ++pos) {
        if (pos == pos1 && blk1 == 0) break;
        const int s = B.sord[(int64_t)b * B.S + pos];
        const int u = B.src_utt[s];
        const int64_t lo = pos == pos0 ? blk0 : 0;
        const int64_t hi = pos == pos1 ? blk1 : B.nblk[u];
        if (lo >= hi) continue;
        f(p, s, u, s - B.src0[u], lo, hi);
        ++p;
    }
}

// True when CTA k of size bucket b has no work.
__device__ __forceinline__ bool chunk_empty(const DevBatch& B, int b, int k) {
    const int64_t o = (int64_t)b * (B.PMAX + 1) + k;
    return B.cta_sp[o] == B.cta_sp[o + 1] && B.cta_b[o] >= B.cta_b[o + 1];
}

// Backward cost model of the partition (relative units measured on GB300 at N =
// 8192, per-CTA times fitted to 2%): a microphone step (one forward transform)
// costs kCostMic, a source step (forward transform, RIR-gradient update, spectral
// products, inverse and dx stores) kCostSrc; a stream also pays kCostFlush per
// RIR-gradient inverse at its end and kCostPiece once.
constexpr int kCostMic = 243;
constexpr int kCostSrc = 562;
constexpr int kCostFlush = 272;
constexpr int kCostPiece = 48;

// Sources per backward stream of each FFT size: the TMEM-accumulator kernels
// (N <= 8192) keep the RIR-gradient spectra of that many sources times two
// microphones in TMEM; the N = 16384 kernel takes one source at a time.
__host__ __device__ constexpr int bwd_src_group(int logN) {
    return logN == 11 ? 8 : logN == 12 ? 4 : logN == 13 ? 4 : 1;
}

// segment s of an utterance with hop h owns the blocks whose start b*h lies
// in [s*seg_len, (s+1)*seg_len)
__host__ __device__ inline void segment_blocks(int64_t s, int64_t seg_len, int64_t hop, int64_t nblk,
                                               int64_t* b0, int64_t* b1) {
    int64_t lo = (s * seg_len + hop - 1) / hop;
    int64_t hi = ((s + 1) * seg_len + hop - 1) / hop;
    if (hi > nblk) hi = nblk;
    *b0 = lo;
    *b1 = hi;
}

// ---------------------------------------------------------------------------
// block reductions (device code of the kernel translation units)
// ---------------------------------------------------------------------------
template <typename Tv, typename Op>
__device__ __forceinline__ Tv warp_reduce(Tv v, Op op) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// result valid in every thread; scratch holds >= 32 elements
template <typename Tv, typename Op>
__device__ __forceinline__ Tv block_reduce(Tv v, Op op, Tv* scratch, Tv ident) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_reduce(v, op);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    Tv r = (threadIdx.x < nw) ? scratch[threadIdx.x] : ident;
    if (wid == 0) r = warp_reduce(r, op);
    if (threadIdx.x == 0) scratch[0] = r;
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

struct OpMaxF { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };
struct OpMaxI { __device__ int operator()(int a, int b) const { return a > b ? a : b; } };
struct OpAddD { __device__ double operator()(double a, double b) const { return a + b; } };
struct OpAddLL { __device__ long long operator()(long long a, long long b) const { return a + b; } };

// ---------------------------------------------------------------------------
// Eq. 7-9: the cut-off of one RIR by one CTA
// ---------------------------------------------------------------------------
// p_th = max h^2 * factor, factor = 10^(-eta/10) computed once on the host in
// FP64.  n_c is the last index whose power is not below p_th (Eq. 8 with its
// strict "<"), and L = min(n_c + 2, Nh) (Eq. 9 keeps one sample beyond n_c).
// The comparison h^2 < p_th is decided exactly in FP64 (h^2 of an FP32 value
// is exact in double and p_th is one rounded product); FP32 bounds settle all
// taps that are clearly above or below so FP64 is used only near p_th.  An
// all-zero RIR keeps L = 1; none != 0 keeps every tap.  tap(i) returns tap i
// (any memory); every thread of the CTA calls it, the result is valid in all
// threads, and with want_frac *frac (valid in thread 0) is the kept share of the
// RIR's energy.  The standalone scan and the fused image-method path both use
// this one function, so they decide alike for equal taps.
struct CutScratch {
    float f[32];
    int i[32];
    double d[32];
};

// Eq. 7-9 for one RIR of n taps read through tap(i), by the CTA: L, and the kept
// energy fraction if asked (in thread 0's *frac).  With KPER > 0 and n <= KPER * blockDim.x every thread
// reads its taps once, all at once, into registers (both passes and the energy sums
// then run there); otherwise each pass reads them again.  The decisions and the
// order of every sum are the same either way.
template <int KPER = 0, typename Tap>
__device__ __forceinline__ int cut_rir(Tap tap, int n, double factor, float sqrt_factor, int none, bool want_frac,
                                       float* frac, CutScratch& cs) {
    const int t = threadIdx.x, nt = blockDim.x;
    constexpr int kC = KPER > 0 ? KPER : 1;
    float c[kC];                                 // the thread's taps i = t + j * nt (in registers)
    const bool inreg = KPER > 0 && n <= KPER * nt;
    float amax = 0.f;
    if (inreg) {
#pragma unroll
        for (int j = 0; j < kC; ++j) {
            const int i = t + j * nt;
            c[j] = i < n ? tap(i) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < kC; ++j) amax = fmaxf(amax, fabsf(c[j]));
    } else {
#pragma unroll 4
        for (int i = t; i < n; i += nt) amax = fmaxf(amax, fabsf(tap(i)));
    }
    amax = block_reduce(amax, OpMaxF(), cs.f, 0.f);
    // P = max h^2 (exact in FP64), p_th = P 10^(-eta/10) in FP64, and FP32 bounds
    // around sqrt(p_th) = max |h| sqrt(factor) that settle the clear taps: with
    // sqrt(factor) rounded to FP32 on the host, the bound's own rounding stays
    // below 3e-7 relative, inside the 1e-6 margin.  Near the FP32 underflow range
    // the bounds open up and every tap goes to the FP64 test.
    const double P = __dmul_rn((double)amax, (double)amax);
    int L;
    if (P == 0.0) {
        L = 1;
    } else if (none) {
        L = n;
    } else {
        const double pth = __dmul_rn(P, factor);
        float tlo = amax * sqrt_factor * (1.f - 1e-6f);   // |h| < tlo   =>  h^2 < p_th
        float thi = amax * sqrt_factor * (1.f + 1e-6f);   // |h| >= thi  =>  h^2 >= p_th
        if (!(tlo > 1e-30f)) {
            tlo = 0.f;
            thi = INFINITY;
        }
        // Eq. 8's test of one tap (FP32 bounds settle the clear ones, FP64 the rest)
        auto keep = [&](float a) {
            if (a < tlo) return false;
            if (a >= thi) return true;
            return !(__dmul_rn((double)a, (double)a) < pth);
        };
        int last = -1;
        if (inreg) {
#pragma unroll
            for (int j = 0; j < kC; ++j) {
                const int i = t + j * nt;
                if (i < n && keep(fabsf(c[j]))) last = i;
            }
        } else {
#pragma unroll 4
            for (int i = t; i < n; i += nt)
                if (keep(fabsf(tap(i)))) last = i;
        }
        last = block_reduce(last, OpMaxI(), cs.i, -1);
        L = last + 2;
        if (L > n) L = n;
    }
    if (want_frac) {
        float et = 0.f, ek = 0.f;
        if (inreg) {
#pragma unroll
            for (int j = 0; j < kC; ++j) {
                const int i = t + j * nt;
                if (i >= n) break;
                const float p = c[j] * c[j];
                et += p;
                if (i < L) ek += p;
            }
        } else {
            for (int i = t; i < n; i += nt) {
                const float v = tap(i);
                const float p = v * v;
                et += p;
                if (i < L) ek += p;
            }
        }
        const double dt = block_reduce((double)et, OpAddD(), cs.d, 0.0);
        const double dk = block_reduce((double)ek, OpAddD(), cs.d, 0.0);
        if (t == 0) *frac = dt > 0.0 ? (float)(dk / dt) : 1.f;
    }
    return L;
}

// ---------------------------------------------------------------------------
// Bounds-checked build (-DRSIM_BOUNDS_CHECK): every store of the kernels' outputs
// and scratch checks its element against the extent of its buffer; an element
// outside latches kErrBounds in the plan's error word (rsim_plan_sync_status
// reports it) and the store is skipped rather than trapping.  The release build
// compiles the checks away.
// ---------------------------------------------------------------------------
#ifdef RSIM_BOUNDS_CHECK
__device__ __forceinline__ bool store_ok(const DevBatch& B, const void* p, const void* base, int64_t bytes) {
    const char* c = static_cast<const char*>(p);
    const char* b = static_cast<const char*>(base);
    const bool ok = b != nullptr && c >= b && c < b + bytes;
    if (!ok) atomicOr(B.err, kErrBounds);
    return ok;
}
#define RSIM_STORE_OK(B, p, base, bytes) ::rsim::store_ok((B), (p), (base), (int64_t)(bytes))
#else
#define RSIM_STORE_OK(B, p, base, bytes) true
#endif
// extents (bytes) of the buffers the kernels write
#define RSIM_Y_BYTES(B) (4 * (B).yoff[(B).U])
#define RSIM_X_BYTES(B) (4 * (B).xoff[(B).S])
#define RSIM_RIR_BYTES(B) (4 * (B).roff[(B).R])

// ---- launchers (defined in the kernel translation units) -------------------
void launch_truncate(const DevBatch& B, const float* rir, double factor, int none,
                     float* energy_kept_frac, int grid, cudaStream_t st);
void launch_power(const DevBatch& B, const float* x, int grid, cudaStream_t st);
void launch_gains(const DevBatch& B, const float* snr_db, float* gains, cudaStream_t st);
void launch_plan(const DevBatch& B, const Queues& Q, cudaStream_t st);
void launch_partition(const DevBatch& B, cudaStream_t st);
// Twiddle tables of one FFT size for 8 and 16 values per thread; every
// tiled kernel picks the table of its own thread shape.
struct Twiddles {
    const float2* e8;
    const float2* e16;
    __host__ __device__ const float2* get(int E) const { return E == 16 ? e16 : e8; }
};
// rir_gain: [R] gain of each RIR folded into its spectrum (per-(i, j) gains), or NULL
void launch_spectrum(int logN, const DevBatch& B, const Queues& Q, const float* rir, const float* rir_gain,
                     float2* Hc, Twiddles tw, int grid, cudaStream_t st);
void launch_forward(int logN, const DevBatch& B, const Queues& Q, const float* x, const float* gains,
                    const float2* Hc, float* y, float* tails, Twiddles tw, int grid,
                    cudaStream_t st);
void launch_fixup(const DevBatch& B, float* y, const float* tails, cudaStream_t st);
// Eq. 1 and the cut-off fused (plans fed by room geometry); see rsim_image.cu
constexpr int kCutMaxTaps = 40960;     // longest RIR the fused path holds in shared memory
int image_cut_grid(int nh_max, int R, int sms);
void launch_image_cut(const DevBatch& B, const rsim_image_geom* geom, int K, float fs, float c0, double factor,
                      int none, int nh_max, float* kept, float* full, float* ekf, int grid, cudaStream_t st);
void launch_backward(int logN, const DevBatch& B, const Queues& Q, const float* g, const float* x,
                     const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                     Twiddles tw, int grid, cudaStream_t st);
// rir_gain non-NULL: per-(i, j) gains; dh scaled per RIR and grad_gains [R] from rir
void launch_finalize(const DevBatch& B, const float* gains, const float* rir_gain, const float* rir,
                     const float* dhp, const float* dap,
                     float* grad_rir, float* grad_gains, cudaStream_t st);

// sets the calling thread's message returned by rsim_last_error()
void set_last_error(const char* msg);

// occupancy helpers (CTAs per SM) and shared-memory sizes of the tiled kernels
int occupancy_spectrum(int logN);
int occupancy_forward(int logN);
int occupancy_backward(int logN);   // CTAs per SM that may run at once (TMEM included)
int threads_for(int logN);
int bwd_threads(int logN);

}  // namespace rsim
