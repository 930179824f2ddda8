// Preparation kernels: RIR tail cut-off (Eq. 7-9), per-source power for the
// SNR gains (Eq. 2's alpha), and the device-side planner that picks the FFT
// size per utterance (Eq. 6) and builds the work queues.
#include "rsim_internal.cuh"

#include <math.h>

namespace rsim {

// ---------------------------------------------------------------------------
// K1: tail cut-off of every RIR (Eq. 7-9), one CTA per RIR (cut_rir)
// ---------------------------------------------------------------------------
constexpr int kTruncThreads = 256;
constexpr int kTruncPer = 64;                    // taps per thread held in registers

__global__ void __launch_bounds__(kTruncThreads, 2)
k_truncate(DevBatch B, const float* __restrict__ rir, double factor, float sqrt_factor, int none,
           float* __restrict__ ekf) {
    __shared__ CutScratch cs;
    for (int r = blockIdx.x; r < B.R; r += gridDim.x) {
        const float* h = rir + B.roff[r];
        const int n = B.rir_len[r];
        float frac;
        // RIRs up to kTruncThreads * kTruncPer taps are read once, into registers
        const int L = cut_rir<kTruncPer>([&](int i) { return __ldg(h + i); }, n, factor, sqrt_factor, none,
                                         ekf != nullptr, &frac, cs);
        if (threadIdx.x == 0) {
            B.L[r] = L;
            if (ekf) ekf[r] = frac;
        }
        __syncthreads();
    }
}

void launch_truncate(const DevBatch& B, const float* rir, double factor, int none,
                     float* energy_kept_frac, int grid, cudaStream_t st) {
    k_truncate<<<grid, kTruncThreads, 0, st>>>(B, rir, factor, (float)sqrt(factor), none, energy_kept_frac);
}

// ---------------------------------------------------------------------------
// K6a: partial sums of x^2 per source, one CTA per 32768-sample chunk
// ---------------------------------------------------------------------------
// Compensated (Kahan) FP32 sums per thread, FP64 across the CTA; the chunk
// partials are added in a fixed order by the planner, so the result does not
// depend on scheduling.
constexpr int kPowThreads = 256;

__global__ void __launch_bounds__(kPowThreads)
k_power(DevBatch B, const float* __restrict__ x) {
    __shared__ double sd[32];
    const int t = threadIdx.x;
    const int64_t total = (int64_t)B.S * B.CH;
    for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
        const int s = (int)(w / B.CH), c = (int)(w % B.CH);
        const int64_t nx = B.n_x[B.src_utt[s]];
        const int64_t c0 = (int64_t)c * kPowerChunk;
        if (c0 >= nx) continue;                 // uniform across the CTA
        const int64_t c1 = (c0 + kPowerChunk < nx) ? c0 + kPowerChunk : nx;
        const float* p = x + B.xoff[s] + c0;
        const int64_t len = c1 - c0;
        // scalar head up to 16-byte alignment, float4 body, scalar tail; four
        // independent compensated sums (one per float4 lane) keep loads in flight
        int64_t head = (int64_t)(((16u - ((uintptr_t)p & 15u)) & 15u) >> 2);
        if (head > len) head = len;
        const int64_t nvec = (len - head) >> 2;
        const int64_t tail0 = head + 4 * nvec;
        float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
        auto acc = [&](int k, float v) {
            const float yv = fmaf(v, v, -comp[k]);
            const float tv = sum[k] + yv;
            comp[k] = (tv - sum[k]) - yv;
            sum[k] = tv;
        };
        for (int64_t i = t; i < head; i += kPowThreads) acc(0, __ldg(p + i));
        for (int64_t i = tail0 + t; i < len; i += kPowThreads) acc(1, __ldg(p + i));
        const float4* p4 = reinterpret_cast<const float4*>(p + head);
        constexpr int kU = 8;                    // float4 loads in flight per thread
        int64_t j = t;
        for (; j + (kU - 1) * kPowThreads < nvec; j += kU * kPowThreads) {
            float4 a[kU];
#pragma unroll
            for (int k = 0; k < kU; ++k) a[k] = __ldg(p4 + j + k * kPowThreads);
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                acc(0, a[k].x); acc(1, a[k].y); acc(2, a[k].z); acc(3, a[k].w);
            }
        }
        for (; j < nvec; j += kPowThreads) {
            const float4 a = __ldg(p4 + j);
            acc(0, a.x); acc(1, a.y); acc(2, a.z); acc(3, a.w);
        }
        double part = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) part += (double)sum[k] - (double)comp[k];
        double d = block_reduce(part, OpAddD(), sd, 0.0);
        if (t == 0) B.pow_part[w] = d;
    }
}

void launch_power(const DevBatch& B, const float* x, int grid, cudaStream_t st) {
    k_power<<<grid, kPowThreads, 0, st>>>(B, x);
}

// ---------------------------------------------------------------------------
// K2a: gains from the source powers (gain modes 0 and 3): alpha_0 = 1,
// alpha_i = sqrt(P_0 / P_i 10^(-SNR_i/10)), P the mean square over [0, Nx).
// Apart from the planner: it needs the power scan, the planner only the cut-off,
// so the planner and the RIR spectra need not wait for the scan.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gains(DevBatch B, const float* __restrict__ snr_db,
                                              float* __restrict__ gains) {
    // one warp per utterance, one source per lane: each lane adds its source's chunk
    // partials in chunk order (FP64), P_0 / P_i is the ratio of those sums (both over
    // the utterance's Nx samples)
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < B.U; u += warps) {
        const int s0 = B.src0[u], I = B.n_src[u];
        // chunks past this utterance's end are never written: sum only the ones that exist
        const int nch = (int)((B.n_x[u] + kPowerChunk - 1) / kPowerChunk);
        double S0 = 0.0;
        for (int i0 = 0; i0 < I; i0 += 32) {
            const int i = i0 + lane;
            double Si = 0.0;
            if (i < I)
                for (int c = 0; c < nch; ++c) Si += B.pow_part[(int64_t)(s0 + i) * B.CH + c];
            if (i0 == 0) S0 = __shfl_sync(0xffffffffu, Si, 0);
            if (i >= I) continue;
            if (i == 0) {
                gains[s0] = 1.f;
            } else if (!(Si > 0.0)) {
                atomicOr(B.err, kErrZeroPower);
                gains[s0 + i] = 0.f;
            } else {
                // the power ratio in FP64, 10^(-SNR/10) and the root in FP32 (an FP64 pow
                // per source is slow on this GPU's FP64 pipe; FP32 keeps alpha within a
                // few 1e-7 relative)
                gains[s0 + i] = sqrtf((float)(S0 / Si) * exp10f(-snr_db[s0 + i] / 10.f));
            }
        }
    }
}

void launch_gains(const DevBatch& B, const float* snr_db, float* gains, cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(((int64_t)B.U * 32 + 255) / 256, 4096);
    k_gains<<<grid > 0 ? grid : 1, 256, 0, st>>>(B, snr_db, gains);
}

// ---------------------------------------------------------------------------
// K2: planner (one CTA)
// ---------------------------------------------------------------------------
// Per utterance: L_max over its RIRs and the FFT size N.
// N minimises the cost of Eq. 6 (ceiling block count, one hop shared by all
// (i, j) of the utterance: hop = N - L_max + 1) weighted by the per-size cost
// table; N must leave hop >= N/4 (a block's tail may then reach several
// blocks ahead; the forward carries it).  An utterance no allowed N fits goes
// to its partitioned path when it has one (no work here), else it is an error.
// Then per FFT size the lists of spectrum jobs (RIRs) and forward tiles
// (segments), in utterance order.  The backward partition of each size is
// k_partition's (below).
constexpr int kPlanThreads = 1024;
constexpr float kConsolidateShare = 0.1f;   // a size below this share of the work is a minority
constexpr float kConsolidateSlack = 0.02f;  // ...and moves if that adds at most this share of the work


__global__ void __launch_bounds__(kPlanThreads)
k_plan(DevBatch B, Queues Q) {
    __shared__ int sm[33];
    const int t = threadIdx.x;
    // ---- FFT size per utterance.  Every thread also tallies, per chosen size m,
    // the predicted work and, per other size d, how much dearer its utterances
    // would be at d (or that some cannot use d) -- for the consolidation below.
    float my_work[kNumBuckets] = {};             // FP32: these only steer a heuristic
    float my_extra[kNumBuckets][kNumBuckets] = {};
    for (int u = t; u < B.U; u += kPlanThreads) {
        int lmax = 1;
        for (int r = B.rir0[u]; r < B.rir0[u + 1]; ++r) lmax = max(lmax, B.L[r]);
        const int64_t nx = B.n_x[u];
        const int I = B.n_src[u], J = B.J;
        float cost[kNumBuckets];
        int best = 0;
        float best_c = 0.f;
        // in a partitioned plan, an utterance the outer planner kept gets no work
        const bool idle = B.active && !B.active[u];
        for (int m = kMinLog; m <= kMaxLog; ++m) {
            cost[m - kMinLog] = -1.f;                  // not allowed or not admissible
            if (idle || !((B.mask >> m) & 1)) continue;
            const int64_t N = 1LL << m;
            const int64_t hop = N - lmax + 1;
            if (4 * hop < N) continue;                 // hop >= N/4 keeps blocks useful
            if (N > B.seg_len) continue;
            const int64_t nb = (nx + hop - 1) / hop;
            const float c = ((float)nb * (I + J) + (float)(I * J)) * B.tuning[m];
            cost[m - kMinLog] = c;
            if (best == 0 || c < best_c) { best = m; best_c = c; }
        }
        // no size fits the kept RIRs: the utterance's partitioned path takes it, if it has one
        const int64_t di = B.defer_idx ? B.defer_idx[u] : -1;
        if (di >= 0) B.defer[di] = best == 0 ? 1 : 0;
        if (best == 0 && di < 0 && !idle) atomicOr(B.err, kErrNoFftSize);
        B.logN[u] = best;
        B.Lmax[u] = lmax;
        if (best) {
#pragma unroll
            for (int b = 0; b < kNumBuckets; ++b) {
                if (best != kMinLog + b) continue;
                my_work[b] += best_c;
#pragma unroll
                for (int d = 0; d < kNumBuckets; ++d) my_extra[b][d] += cost[d] < 0.f ? 1e30f : cost[d] - best_c;
            }
        }
    }
    // fixed-order block sums (warp shuffles, then the warps' partials in order)
    {
        constexpr int kVals = kNumBuckets * (kNumBuckets + 1);
        __shared__ float part[kVals][kPlanThreads / 32];
        __shared__ float sums[kVals];
        const int lane = t & 31, wid = t >> 5;
#pragma unroll
        for (int q = 0; q < kVals; ++q) {
            float v = q < kNumBuckets ? my_work[q]
                                       : my_extra[(q - kNumBuckets) / kNumBuckets][(q - kNumBuckets) % kNumBuckets];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[q][wid] = v;
        }
        __syncthreads();
        if (t < kVals) {
            float v = 0.f;
            for (int w = 0; w < kPlanThreads / 32; ++w) v += part[t][w];
            sums[t] = v;
        }
        __syncthreads();
        // consolidation: a size carrying under kConsolidateShare of the predicted work
        // runs as a small launch beside the dominant one and finishes late (its CTAs
        // queue behind the persistent ones); all its utterances move to the dominant
        // size when every one of them fits it and together they cost at most
        // kConsolidateSlack of the batch's predicted work more there
        if (t == 0) {
            int dom = 0;
            float tot = 0.f;
            for (int b = 0; b < kNumBuckets; ++b) {
                tot += sums[b];
                if (sums[b] > sums[dom]) dom = b;
            }
            int moved = 0;
            for (int b = 0; b < kNumBuckets; ++b)
                if (b != dom && sums[b] > 0.f && sums[b] < kConsolidateShare * tot &&
                    sums[kNumBuckets + b * kNumBuckets + dom] < kConsolidateSlack * tot)
                    moved |= 1 << b;
            sm[32] = dom;
            sm[31] = moved;
        }
        __syncthreads();
    }
    const int dom_m = kMinLog + sm[32], moved = sm[31];
    for (int u = t; u < B.U; u += kPlanThreads) {
        int m = B.logN[u];
        if (m != 0 && ((moved >> (m - kMinLog)) & 1)) m = dom_m;
        B.logN[u] = m;
        const int64_t nx = B.n_x[u];
        const int64_t hop = m ? (1LL << m) - B.Lmax[u] + 1 : 1;
        B.hop[u] = (int)hop;
        B.nblk[u] = m ? (int)((nx + hop - 1) / hop) : 0;
    }
    __syncthreads();
    const int per = (B.U + kPlanThreads - 1) / kPlanThreads;
    const int u0 = min(B.U, t * per), u1 = min(B.U, u0 + per);
    const int lane = t & 31, wid = t >> 5;
    // ---- work lists.  The forward's tiles go dearest first (cost: the tile's blocks x
    // (I + J) transforms, in kFwdCls classes of equal width up to a bound on the dearest
    // tile), so that the persistent CTAs end on cheap tiles (longest-processing-time
    // first), which shortens the launch's ragged end: a shared-memory histogram of the
    // (size, class) pairs, then each utterance takes the next run of slots of each of
    // its pairs (the order of the runs within a class is that of the slot claims;
    // results do not depend on it).  The
    // spectrum lists: one contiguous chunk of utterances per thread, laid out by a
    // block-wide exclusive scan of the per-thread counts.
    constexpr int kFwdCls = 8;
    // the tile's blocks in FP32 (only the order depends on them; the tiles' own block
    // ranges are computed exactly where they are processed)
    auto tile_cost = [&](int u, int g) {
        const float r = (float)B.seg_len / (float)B.hop[u], nb = (float)B.nblk[u];
        const float s = (float)(g - B.seg0[u]);
        const float b0 = fminf(ceilf(s * r), nb), b1 = fminf(ceilf((s + 1.f) * r), nb);
        return (int)(b1 - b0) * (B.n_src[u] + B.J);
    };
    int cmax = 0;                                // a tile holds at most ceil(seg_len / hop) + 1 blocks
    for (int u = u0; u < u1; ++u)
        if (B.logN[u] != 0)
            cmax = max(cmax, (int)((B.seg_len + B.hop[u] - 1) / B.hop[u] + 1) * (B.n_src[u] + B.J));
    cmax = block_reduce(cmax, OpMaxI(), sm, 0);
    auto tile_cls = [&](int c) { return (int)((int64_t)(cmax - min(c, cmax)) * kFwdCls / (cmax + 1)); };
    __shared__ int hist[kNumBuckets * kFwdCls];
    if (t < kNumBuckets * kFwdCls) hist[t] = 0;
    __syncthreads();
    for (int u = u0; u < u1; ++u) {
        const int m = B.logN[u];
        if (m == 0) continue;
        for (int g = B.seg0[u]; g < B.seg0[u + 1]; ++g)
            atomicAdd(&hist[(m - kMinLog) * kFwdCls + tile_cls(tile_cost(u, g))], 1);
    }
    __syncthreads();
    if (t < kNumBuckets) {                       // class c of size t starts after the dearer ones
        int acc = 0;
        for (int c = 0; c < kFwdCls; ++c) {
            const int v = hist[t * kFwdCls + c];
            hist[t * kFwdCls + c] = acc;
            acc += v;
        }
        Q.count[Q.idx(kListFwd, t)] = acc;
    }
    __syncthreads();
    // each utterance claims its tiles of a class as one run of slots, so that an
    // utterance's tiles stay together in the list (its RIR spectra then serve
    // neighbouring CTAs from L2)
    for (int u = u0; u < u1; ++u) {
        const int m = B.logN[u];
        if (m == 0) continue;
        int n[kFwdCls];
#pragma unroll
        for (int c = 0; c < kFwdCls; ++c) n[c] = 0;
        for (int g = B.seg0[u]; g < B.seg0[u + 1]; ++g) {
            const int c = tile_cls(tile_cost(u, g));
#pragma unroll
            for (int q = 0; q < kFwdCls; ++q) n[q] += q == c;
        }
#pragma unroll
        for (int q = 0; q < kFwdCls; ++q)
            if (n[q]) n[q] = atomicAdd(&hist[(m - kMinLog) * kFwdCls + q], n[q]);
        int32_t* lf = Q.lst(kListFwd, m - kMinLog);
        for (int g = B.seg0[u]; g < B.seg0[u + 1]; ++g) {
            const int c = tile_cls(tile_cost(u, g));
            int pos = 0;
#pragma unroll
            for (int q = 0; q < kFwdCls; ++q)
                if (q == c) pos = n[q]++;
            lf[pos] = g;
        }
    }
    int cnt[kNumBuckets];
#pragma unroll
    for (int q = 0; q < kNumBuckets; ++q) cnt[q] = 0;
    for (int u = u0; u < u1; ++u) {
        const int m = B.logN[u];
        if (m == 0) continue;
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q)
            if (q == m - kMinLog) cnt[q] += B.rir0[u + 1] - B.rir0[u];
    }
    __shared__ int wtot[kPlanThreads / 32][kNumBuckets];
    __shared__ int ltot[kNumBuckets];
    int off[kNumBuckets];
    {
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) {
            int incl = cnt[q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += n;
            }
            off[q] = incl - cnt[q];
            if (lane == 31) wtot[wid][q] = incl;
        }
        __syncthreads();
        if (t < kNumBuckets) {                   // exclusive scan of the warps' totals
            int acc = 0;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                const int v = wtot[w][t];
                wtot[w][t] = acc;
                acc += v;
            }
            ltot[t] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) off[q] += wtot[wid][q];
    }
    for (int u = u0; u < u1; ++u) {
        const int m = B.logN[u];
        if (m == 0) continue;
        int32_t* ls = Q.lst(kListSpec, m - kMinLog);
        int os = 0;
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) {
            if (q != m - kMinLog) continue;
            os = off[q];
            off[q] += B.rir0[u + 1] - B.rir0[u];
        }
        for (int r = B.rir0[u]; r < B.rir0[u + 1]; ++r) ls[os++] = r;
    }
    if (t < kNumBuckets) {
        Q.count[Q.idx(kListSpec, t)] = ltot[t];
        Q.count[Q.idx(kListBwd, t)] = 0;
        Q.next[Q.idx(kListFwd, t)] = 0;
        Q.next[Q.idx(kListBwd, t)] = 0;
        Q.next[Q.idx(kListSpec, t)] = 0;
    }
}


// ---------------------------------------------------------------------------
// K2b: the backward partition (one CTA), from the sizes and block counts the
// planner chose.  Only the backward and its finalizer read what it writes, so
// it runs beside the spectra and the forward.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPlanThreads)
k_partition(DevBatch B) {
    __shared__ long long pw_scratch[32];
    const int t = threadIdx.x;
    const int per = (B.U + kPlanThreads - 1) / kPlanThreads;
    const int u0 = min(B.U, t * per), u1 = min(B.U, u0 + per);
    const int ngrp_j = (B.J + kJG - 1) / kJG;
    const int lane = t & 31, wid = t >> 5;
    // cost of one block of a stream of ig sources, and of the whole stream (its
    // blocks, then the flush of its RIR-gradient accumulators)
    auto block_cost = [&](int ig) { return kCostMic * B.J + kCostSrc * ngrp_j * ig; };
    auto stream_total = [&](int nb, int ig) {
        return (long long)nb * block_cost(ig) + (long long)kCostFlush * ig * B.J + kCostPiece;
    };
    // ---- backward partition, step 1: the streams of each size in batch order and the
    // exclusive prefix of their costs (utterances in contiguous chunks per thread)
    {
        int ns[kNumBuckets];
        long long cs[kNumBuckets];
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) { ns[q] = 0; cs[q] = 0; }
        for (int u = u0; u < u1; ++u) {
            const int m = B.logN[u];
            if (m == 0) continue;
            const int sg = bwd_src_group(m), I = B.n_src[u];
#pragma unroll
            for (int q = 0; q < kNumBuckets; ++q) {
                if (q != m - kMinLog) continue;
                for (int i0 = 0; i0 < I; i0 += sg) {
                    ns[q] += 1;
                    cs[q] += stream_total(B.nblk[u], min(sg, I - i0));
                }
            }
        }
        __shared__ int wn[kPlanThreads / 32][kNumBuckets];
        __shared__ long long wc[kPlanThreads / 32][kNumBuckets];
        int on[kNumBuckets];
        long long oc[kNumBuckets];
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) {
            int in = ns[q];
            long long ic = cs[q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n1 = __shfl_up_sync(0xffffffffu, in, o);
                const long long c1 = __shfl_up_sync(0xffffffffu, ic, o);
                if (lane >= o) { in += n1; ic += c1; }
            }
            on[q] = in - ns[q];
            oc[q] = ic - cs[q];
            if (lane == 31) { wn[wid][q] = in; wc[wid][q] = ic; }
        }
        __syncthreads();
        if (t < kNumBuckets) {                    // exclusive scan of the warps' totals
            int an = 0;
            long long ac = 0;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                const int vn = wn[w][t];
                const long long vc = wc[w][t];
                wn[w][t] = an;
                wc[w][t] = ac;
                an += vn;
                ac += vc;
            }
            B.nstream[t] = an;
            B.spre[(int64_t)t * (B.S + 1) + an] = ac;   // the size's total cost
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kNumBuckets; ++q) { on[q] += wn[wid][q]; oc[q] += wc[wid][q]; }
        for (int u = u0; u < u1; ++u) {
            const int m = B.logN[u];
            if (m == 0) continue;
            const int sg = bwd_src_group(m), I = B.n_src[u];
#pragma unroll
            for (int q = 0; q < kNumBuckets; ++q) {
                if (q != m - kMinLog) continue;
                for (int i0 = 0; i0 < I; i0 += sg) {
                    B.sord[(int64_t)q * B.S + on[q]] = B.src0[u] + i0;
                    B.spre[(int64_t)q * (B.S + 1) + on[q]] = oc[q];
                    on[q] += 1;
                    oc[q] += stream_total(B.nblk[u], min(sg, I - i0));
                }
            }
        }
    }
    __syncthreads();
    // per-block cost of the stream at position pos of size q
    auto stream_cost = [&](int q, int pos, int* u_out) {
        const int sidx = B.sord[(int64_t)q * B.S + pos];
        const int u = B.src_utt[sidx];
        const int sg = bwd_src_group(kMinLog + q);
        *u_out = u;
        return block_cost(min(sg, B.n_src[u] - (sidx - B.src0[u])));
    };
    // ---- step 2: the kept taps of the RIRs before each one (exclusive prefix over the
    // batch, RIRs in contiguous chunks per thread): a piece's RIR-gradient partials
    // hold its stream's kept taps
    {
        const int rper = (B.R + kPlanThreads - 1) / kPlanThreads;
        const int r0t = min(B.R, t * rper), r1t = min(B.R, r0t + rper);
        long long mine = 0;
        for (int r = r0t; r < r1t; ++r) mine += B.L[r];
        __shared__ long long lw[kPlanThreads / 32];
        long long incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) lw[wid] = incl;
        __syncthreads();
        if (t == 0) {
            long long acc = 0;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                const long long v = lw[w];
                lw[w] = acc;
                acc += v;
            }
            B.lpre[B.R] = acc;
        }
        __syncthreads();
        long long run = incl - mine + lw[wid];
        for (int r = r0t; r < r1t; ++r) {
            B.lpre[r] = run;
            run += B.L[r];
        }
    }
    __syncthreads();
    // ---- steps 3 and 4, repeated until the partials fit: where each CTA's chunk
    // starts, then the pieces.  CTA k of size q (k < P, P the CTAs that take work)
    // starts at the first block whose cost position is at least ceil(k T / P) (a
    // position inside a stream's flush is its end); CTAs from P on, and the end
    // sentinel, get (streams, 0).  Every CTA boundary inside a stream adds a piece
    // holding a copy of the stream's partials; when all of them exceed the
    // RIR-gradient partials, every size's P is halved and the cut is redone (at
    // P = 1 the pieces are the streams, which always fit).
    const int PM = B.PMAX + 1;
    __shared__ int peff[kNumBuckets];
    __shared__ long long dtot;
    if (t < kNumBuckets) peff[t] = B.bgrid[t];
    __syncthreads();
    auto walk = [&](int q, int k, auto visit) {
        const int pos0 = B.cta_sp[(int64_t)q * PM + k], blk0 = B.cta_b[(int64_t)q * PM + k];
        const int pos1 = B.cta_sp[(int64_t)q * PM + k + 1], blk1 = B.cta_b[(int64_t)q * PM + k + 1];
        for (int pos = pos0; pos <= pos1; ++pos) {
            if (pos == pos1 && blk1 == 0) break;
            const int sidx = B.sord[(int64_t)q * B.S + pos];
            const int u = B.src_utt[sidx];
            const int lo = pos == pos0 ? blk0 : 0;
            const int hi = pos == pos1 ? blk1 : B.nblk[u];
            if (lo >= hi) continue;
            const int i0 = sidx - B.src0[u];
            const int ig = min(bwd_src_group(kMinLog + q), B.n_src[u] - i0);
            const int r0 = B.rir0[u] + i0 * B.J;
            const long long taps = B.lpre[r0 + ig * B.J] - B.lpre[r0];
            visit(sidx, lo == 0, hi == B.nblk[u], taps);
        }
    };
    const int NE = kNumBuckets * PM;
    const int pe = (NE + kPlanThreads - 1) / kPlanThreads;
    const int e0 = min(NE, t * pe), e1 = min(NE, e0 + pe);
    for (;;) {
        // step 3: chunk starts
        for (int idx = t; idx < kNumBuckets * PM; idx += kPlanThreads) {
            const int q = idx / PM, k = idx - q * PM;
            const int P = peff[q];
            if (k > B.bgrid[q]) continue;
            const int n = B.nstream[q];
            const int64_t* pre = B.spre + (int64_t)q * (B.S + 1);
            int pos = n, blk = 0;
            if (k < P && n > 0) {
                const long long T = pre[n];
                const long long x = (T * k + P - 1) / P;
                int lo = 0, hi = n;               // largest pos < n with pre[pos] <= x
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid] <= x) lo = mid; else hi = mid;
                }
                int u;
                const int c = stream_cost(q, lo, &u);
                const long long bk = (x - pre[lo] + c - 1) / c;
                if (bk >= B.nblk[u]) { pos = lo + 1; blk = 0; }
                else { pos = lo; blk = (int)bk; }
            }
            B.cta_sp[(int64_t)q * PM + k] = pos;
            B.cta_b[(int64_t)q * PM + k] = blk;
        }
        __syncthreads();
        // step 4a: the partials all pieces need
        long long nd = 0;
        for (int e = e0; e < e1; ++e) {
            const int q = e / PM, k = e - q * PM;
            if (k < B.bgrid[q]) walk(q, k, [&](int, bool, bool, long long taps) { nd += taps; });
        }
        nd = block_reduce(nd, OpAddLL(), reinterpret_cast<long long*>(pw_scratch), 0LL);
        if (t == 0) dtot = nd;
        __syncthreads();
        bool done = dtot <= B.NDHP;
        if (!done) {
            bool all_one = true;
            for (int q = 0; q < kNumBuckets; ++q) all_one = all_one && peff[q] <= 1;
            done = all_one;                       // cannot happen: single chunks fit
        }
        if (done) break;
        __syncthreads();
        if (t < kNumBuckets) peff[t] = max(1, peff[t] / 2);
        __syncthreads();
    }
    // step 4b: number the pieces in (size, CTA) order, write their partial offsets and
    // mark the first and last piece of every stream
    {
        int np = 0;
        long long nd = 0;
        for (int e = e0; e < e1; ++e) {
            const int q = e / PM, k = e - q * PM;
            if (k < B.bgrid[q]) walk(q, k, [&](int, bool, bool, long long taps) { np += 1; nd += taps; });
        }
        __shared__ int pw[kPlanThreads / 32];
        __shared__ long long dw[kPlanThreads / 32];
        int ip = np;
        long long id = nd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n1 = __shfl_up_sync(0xffffffffu, ip, o);
            const long long d1 = __shfl_up_sync(0xffffffffu, id, o);
            if (lane >= o) { ip += n1; id += d1; }
        }
        if (lane == 31) { pw[wid] = ip; dw[wid] = id; }
        __syncthreads();
        if (t == 0) {
            int an = 0;
            long long ad = 0;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                const int vn = pw[w];
                const long long vd = dw[w];
                pw[w] = an;
                dw[w] = ad;
                an += vn;
                ad += vd;
            }
        }
        __syncthreads();
        int p = ip - np + pw[wid];
        long long d = id - nd + dw[wid];
        for (int e = e0; e < e1; ++e) {
            const int q = e / PM, k = e - q * PM;
            if (k >= B.bgrid[q]) continue;
            B.cta_p[(int64_t)q * PM + k] = p;
            walk(q, k, [&](int sidx, bool first, bool last, long long taps) {
                B.piece_dh[p] = d;
                if (first) B.s_first[sidx] = p;
                if (last) B.s_last[sidx] = p;
                p += 1;
                d += taps;
            });
        }
    }
}

void launch_plan(const DevBatch& B, const Queues& Q, cudaStream_t st) {
    k_plan<<<1, kPlanThreads, 0, st>>>(B, Q);
}

void launch_partition(const DevBatch& B, cudaStream_t st) {
    k_partition<<<1, kPlanThreads, 0, st>>>(B);
}

}  // namespace rsim
