// Forward path: RIR spectra (computed once per RIR, Sec. 2.2), the fused
// overlap-add filter-and-mix (Eq. 2 evaluated block by block as in Eq. 6),
// and the fix-up that joins output blocks across tile boundaries.
#include "rsim_fft.cuh"
#include "rsim_internal.cuh"

namespace rsim {

// Pops the next job index of a persistent kernel's queue (same value in all
// threads).  Returns -1 when the queue is drained.
__device__ __forceinline__ int pop_job(const Queues& Q, int kind, int b, int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int i = atomicAdd(&Q.next[Q.idx(kind, b)], 1);
        *slot = (i < Q.count[Q.idx(kind, b)]) ? Q.lst(kind, b)[i] : -1;
    }
    __syncthreads();
    return *slot;
}

// ---------------------------------------------------------------------------
// K3: Hc_r = rFFT_N(hhat_r) / N in pair layout order (slot 0 = (H[0], H[N/2]))
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(M / e_for(M))
k_spectrum(DevBatch B, Queues Q, int bucket, const float* __restrict__ rir, const float* __restrict__ rir_gain,
           float2* __restrict__ Hc, const float2* __restrict__ tw) {
    constexpr int E = e_for(M);
    constexpr int T = M / E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    __shared__ int slot;
    const int t = threadIdx.x;
    const float inv_n = 1.0f / (2.0f * M);
    for (;;) {
        const int r = pop_job(Q, kListSpec, bucket, &slot);
        if (r < 0) break;
        float2 P[E];
        rfft_pairs<M, E>(P, rir + B.roff[r], B.L[r], sm, tw, t);
        const float sc = rir_gain ? inv_n * rir_gain[r] : inv_n;   // a per-(i, j) gain folds in here
        // mirror pairs side by side: slot k < M/2 holds (H[k], H[M-k]); slot 0 holds
        // ((H[0], H[N/2]) packed, H[M/2])
        float4* H = reinterpret_cast<float4*>(Hc + (int64_t)r * B.MMAX);
#pragma unroll
        for (int s = 0; s < E / 2; ++s) {
            const float2 a = cscale(P[2 * s], sc), c = cscale(P[2 * s + 1], sc);
            if (RSIM_STORE_OK(B, &H[t + s * T], Hc, (int64_t)B.R * B.MMAX * sizeof(float2)))
                H[t + s * T] = make_float4(a.x, a.y, c.x, c.y);
        }
    }
}

// ---------------------------------------------------------------------------
// K4: fused overlap-add filter-and-mix, persistent over segment tiles
// ---------------------------------------------------------------------------
// For each block b of the tile's segment (hop = N - L_max + 1):
//   X_i = rFFT_N(x_i[b hop, b hop + hop))                 for every source i
//   Y_j = sum_i alpha_i Hc_ij X_i                          split fused with the
//                                                          MAC, Y_j in registers
//   y_j block = irFFT_N(Y_j) plus the carry of the earlier blocks; its first
//   hop samples are stored, the last L_max - 1 samples are the new carry.
// The next source's x block is prefetched one step ahead by one bulk copy
// into a shared-memory stage (whole 16-byte chunks by the copy engine,
// completing on an mbarrier the threads wait on with a bounded wait) while the
// current one is transformed; the RIR spectra are read through L2 as mirror
// pairs.  Twiddles are copied to shared memory once per CTA (N <= 8192).  The tail leaving the segment's last
// block goes to `tails`; the tile of the next segment stored its first block
// without it and k_fixup adds it afterwards (one FP32 add, the same one done
// in-tile, so results do not depend on the segmentation).  Microphones are
// processed in groups of kJG; source spectra are recomputed per group.
// Thread shape and shared-memory layout of the forward kernel per size:
// E values per thread (T = M / E threads), whether the carried tails and the
// twiddles sit in shared memory, and the CTAs per SM the register budget is
// set for.
template <int M>
struct FwdCfg {
    static constexpr int E = (M == 4096 || M == 8192) ? 16 : 8;
    static constexpr int T = M / E;
    static constexpr int kMinBlocks = (M <= 4096) ? 2 : 1;
    static constexpr bool kTailSmem = (M <= 2048);
    static constexpr bool kTwSmem = (M <= 4096);
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_sm = 0;
    static constexpr size_t o_xs = a16(o_sm + sizeof(float2) * padded_len(M));
    static constexpr size_t o_tl = a16(o_xs + sizeof(float) * (2 * M + 8));   // + chunk offset room
    static constexpr size_t o_tw = a16(o_tl + (kTailSmem ? sizeof(float) * kJG * 2 * M : 0));
    static constexpr size_t bytes = a16(o_tw + (kTwSmem ? sizeof(float2) * FftPlan<M, E>::TW_LEN : 0));
};

template <int M>
__global__ void __launch_bounds__(FwdCfg<M>::T, FwdCfg<M>::kMinBlocks)
k_forward(DevBatch B, Queues Q, int bucket, const float* __restrict__ x,
          const float* __restrict__ gains, const float2* __restrict__ Hc, float* __restrict__ y,
          float* __restrict__ tails, const float2* __restrict__ twg) {
    using L = FwdCfg<M>;
    constexpr int E = L::E;
    constexpr int T = M / E;
    using Pl = FftPlan<M, E>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw + L::o_sm);
    float* xs = reinterpret_cast<float*>(smem_raw + L::o_xs);
    float* tl_smem = reinterpret_cast<float*>(smem_raw + L::o_tl);
    __shared__ int slot;
    __shared__ __align__(8) uint64_t mbar;
    // the tile's per-source gains and offsets and its utterance's output offset, read once
    // per tile (every source step reads them: from global memory each read would sit on
    // the step's path)
    // (up to kMaxPartSources: a partitioned plan's utterances hold that many virtual sources)
    constexpr int kSrc = kMaxPartSources > kMaxSources ? kMaxPartSources : kMaxSources;
    __shared__ float f_gain[kSrc];
    __shared__ int64_t f_xoff[kSrc], f_xso[kSrc];
    __shared__ int64_t f_yoff;
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&mbar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t ph = 0;                             // parity of the stage's next phase
    int xoff = 0;                                // float offset of the data in the stage
    bool bad = false;                            // a bounded wait ran out (no new copies then)
    const float2* tw = twg;
    if constexpr (L::kTwSmem) {
        float2* tws = reinterpret_cast<float2*>(smem_raw + L::o_tw);
        for (int k = t; k < Pl::TW_LEN; k += T) tws[k] = twg[k];
        __syncthreads();
        tw = tws;
    }
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    for (;;) {
        const int g = pop_job(Q, kListFwd, bucket, &slot);
        if (g < 0) break;
        const int u = B.seg_utt[g];
        const int64_t s = g - B.seg0[u];
        const int64_t nx = B.n_x[u];
        const int64_t ny = B.n_y[u];
        const int hop = B.hop[u];
        const int tail_len = B.Lmax[u] - 1;
        // end of the convolution's support (the full output is zero from here on)
        const int64_t ye = min(ny, nx + (int64_t)tail_len);
        int64_t b0, b1;
        segment_blocks(s, B.seg_len, hop, B.nblk[u], &b0, &b1);
        if (b0 >= b1) continue;
        const int I = B.n_src[u], J = B.J;
        const int sb = B.src0[u], rb = B.rir0[u];
        // (the previous tile ended on a barrier; these are read after the group's first one)
        for (int q = t; q < I; q += T) {
            f_gain[q] = __ldg(gains + sb + q);
            f_xoff[q] = B.xoff[sb + q];
            f_xso[q] = B.xspec ? B.xspec_off[sb + q] : 0;
        }
        if (t == 0) f_yoff = B.yoff[u];
        for (int j0 = 0; j0 < J; j0 += kJG) {
            const int jn = min(kJG, J - j0);
            // one bulk copy per source block into the stage (whole 16-byte chunks by
            // the copy engine, completing on mbar; ragged ends and zeros by stores)
            auto stage_x = [&](int64_t b, int i) {
                if (bad) return;
                const int64_t p = b * hop;
                xoff = stage_real_bulk<M, E>(xs, x + f_xoff[i] + p, min((int64_t)hop, nx - p), &mbar, t,
                                             B.test_withhold != 0);
            };
            // carried tail of mic jj: shared memory, or this tile's slot of `tails`
            auto tl = [&](int jj) -> float* {
                if constexpr (L::kTailSmem) return tl_smem + jj * 2 * M;
                else return tails + ((int64_t)g * J + j0 + jj) * 2 * B.MMAX;
            };
            const int64_t tails_bytes = (int64_t)B.NSEG * J * 2 * B.MMAX * sizeof(float);
            // a store into a carried tail: shared memory, or checked against `tails`
            auto tail_ok = [&](const float* q) {
                if constexpr (L::kTailSmem) return true;
                else return RSIM_STORE_OK(B, q, tails, tails_bytes);
            };
            const int64_t y_bytes = RSIM_Y_BYTES(B);
            __syncthreads();                     // stages and tails are free
            for (int jj = 0; jj < jn; ++jj)
                for (int n = t; n < tail_len; n += T)
                    if (tail_ok(tl(jj) + n)) tl(jj)[n] = 0.f;
            stage_x(b0, 0);
            for (int64_t b = b0; b < b1; ++b) {
                const int64_t pos = b * hop;
                float2 Y[kJG][E];
#pragma unroll
                for (int jj = 0; jj < kJG; ++jj)
#pragma unroll
                    for (int e = 0; e < E; ++e) Y[jj][e] = make_float2(0.f, 0.f);
                for (int i = 0; i < I; ++i) {
                    // x_i is in
                    if (!bad && !mbar_wait_bounded(&mbar, ph)) {
                        mbar_wait_bounded(&mbar, ph, 100000000ull);   // one more chance to land
                        bad = true;
                    }
                    ph ^= 1u;
                    __syncthreads();
                    float2 v[E];
                    load_staged_at<M, E>(v, xs, xoff, t);
                    __syncthreads();             // xs fully read: reuse it
                    if (i + 1 < I) stage_x(b, i + 1);
                    else if (b + 1 < b1) stage_x(b + 1, 0);
                    fft_core<M, E>(v, sm, tw, t);
                    __syncthreads();
                    store_strided<M, E>(v, sm, t);
                    __syncthreads();
                    const float a = f_gain[i];
                    const float2* H0 = Hc + (int64_t)(rb + i * J + j0) * B.MMAX;
                    // the block's spectrum, kept for the backward (first microphone group)
                    float4* xsp = nullptr;
                    {
                        if (B.xspec && j0 == 0)
                            xsp = reinterpret_cast<float4*>(reinterpret_cast<char*>(B.xspec) + f_xso[i]) +
                                  b * (M / 2);
                    }
#pragma unroll
                    for (int q = 0; q < E / 2; ++q) {
                        const int k = t + q * T;
                        float2 xa, xb;
                        split_pair<M>(sm, wsplit, k, xa, xb);
                        // streaming store: read once, by the backward, so it should not evict
                        // the RIR spectra this kernel keeps re-reading from L2
                        if (xsp && RSIM_STORE_OK(B, xsp + k, B.xspec, B.xspec_bytes))
                            __stcs(xsp + k, make_float4(xa.x, xa.y, xb.x, xb.y));
                        xa = cscale(xa, a);
                        xb = cscale(xb, a);
#pragma unroll
                        for (int jj = 0; jj < kJG; ++jj) {
                            if (jj >= jn) break;
                            const float4 hh = __ldg(reinterpret_cast<const float4*>(H0 + (int64_t)jj * B.MMAX) + k);
                            const float2 ha = make_float2(hh.x, hh.y), hb = make_float2(hh.z, hh.w);
                            if (k == 0) {            // slot 0 holds two real bins
                                Y[jj][0].x += xa.x * ha.x;
                                Y[jj][0].y += xa.y * ha.y;
                            } else {
                                Y[jj][2 * q] = cadd(Y[jj][2 * q], cmul(xa, ha));
                            }
                            Y[jj][2 * q + 1] = cadd(Y[jj][2 * q + 1], cmul(xb, hb));
                        }
                    }
                }
#pragma unroll
                for (int jj = 0; jj < kJG; ++jj) {
                    if (jj >= jn) break;
                    float2 v[E];
                    irfft_pairs<M, E>(v, Y[jj], sm, tw, t);
                    float* yj = y + f_yoff + (int64_t)(j0 + jj) * ny + pos;
                    float* tlj = tl(jj);
                    const int64_t lim = ye - pos;
                    // every sample n < N of the block adds the carried sum at n;
                    // [0, hop) is stored, [hop, N) becomes the new carry (which
                    // reaches several blocks ahead when L_max - 1 > hop)
                    const int ilim = (int)min((int64_t)hop, lim);
                    const bool pairs = (reinterpret_cast<uintptr_t>(yj) & 7) == 0;
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
                        if (n < tail_len) v[q].x += tlj[n];
                        if (n + 1 < tail_len) v[q].y += tlj[n + 1];
                        if (pairs && n + 1 < ilim) {
                            if (RSIM_STORE_OK(B, yj + n + 1, y, y_bytes)) *reinterpret_cast<float2*>(yj + n) = v[q];
                        } else {
                            if (n < ilim && RSIM_STORE_OK(B, yj + n, y, y_bytes)) yj[n] = v[q].x;
                            if (n + 1 < ilim && RSIM_STORE_OK(B, yj + n + 1, y, y_bytes)) yj[n + 1] = v[q].y;
                        }
                    }
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
                        if (n >= hop && n - hop < tail_len && tail_ok(tlj + n - hop)) tlj[n - hop] = v[q].x;
                        if (n + 1 >= hop && n + 1 - hop < tail_len && tail_ok(tlj + n + 1 - hop))
                            tlj[n + 1 - hop] = v[q].y;
                    }
                }
            }
            if constexpr (L::kTailSmem) {
                __syncthreads();
                for (int jj = 0; jj < jn; ++jj) {
                    float* dst = tails + ((int64_t)g * J + j0 + jj) * 2 * B.MMAX;
                    for (int n = t; n < tail_len; n += T)
                        if (RSIM_STORE_OK(B, dst + n, tails, tails_bytes)) dst[n] = tl(jj)[n];
                }
            }
            if (ny > nx && b1 == B.nblk[u]) {
                // full output: the carry past the last block is the end of the
                // convolution (up to Nx + L_max - 1), then exact zeros
                __syncthreads();
                const int64_t end = b1 * hop;
                for (int jj = 0; jj < jn; ++jj) {
                    float* yj = y + B.yoff[u] + (int64_t)(j0 + jj) * ny;
                    for (int64_t n = min(end, ye) + t; n < ny; n += T)
                        if (RSIM_STORE_OK(B, yj + n, y, y_bytes)) yj[n] = (n < ye) ? tl(jj)[n - end] : 0.f;
                }
            }
        }
        if (__syncthreads_or(bad)) {             // a copy never completed: report and stop
            if (t == 0) atomicOr(B.err, kErrWaitTimeout);
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// K5: add each segment's incoming tail to its first block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_fixup(DevBatch B, float* __restrict__ y, const float* __restrict__ tails) {
    const int j = blockIdx.y;                    // one microphone per grid row
    for (int g = blockIdx.x; g < B.NSEG; g += gridDim.x) {
        const int u = B.seg_utt[g];
        const int64_t s = g - B.seg0[u];
        if (s == 0 || B.logN[u] == 0) continue;
        const int hop = B.hop[u];
        int64_t b0, b1;
        segment_blocks(s, B.seg_len, hop, B.nblk[u], &b0, &b1);
        if (b0 >= b1) continue;
        const int64_t ny = B.n_y[u];
        const int64_t pos = b0 * hop;
        const int tail_len = B.Lmax[u] - 1;
        const int64_t ye = min(ny, B.n_x[u] + (int64_t)tail_len);
        const int lim = (int)min((int64_t)tail_len, ye - pos);
        // eight independent read-add-write rounds in flight per thread
        constexpr int kU = 8;
        const float* src = tails + ((int64_t)(g - 1) * B.J + j) * 2 * B.MMAX;
        float* yj = y + B.yoff[u] + (int64_t)j * ny + pos;
        for (int n0 = threadIdx.x; n0 < lim; n0 += kU * blockDim.x) {
            float a[kU], c[kU];
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int n = n0 + k * blockDim.x;
                a[k] = n < lim ? yj[n] : 0.f;
                c[k] = n < lim ? src[n] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int n = n0 + k * blockDim.x;
                if (n < lim && RSIM_STORE_OK(B, yj + n, y, RSIM_Y_BYTES(B))) yj[n] = a[k] + c[k];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int M>
constexpr int smem_spectrum() { return (int)sizeof(float2) * padded_len(M); }
template <int M>
constexpr int smem_forward() { return (int)FwdCfg<M>::bytes; }

template <int M>
static void spectrum_m(const DevBatch& B, const Queues& Q, int bucket, const float* rir, const float* rir_gain,
                       float2* Hc, Twiddles tw, int grid, cudaStream_t st) {
    k_spectrum<M><<<grid, M / e_for(M), smem_spectrum<M>(), st>>>(B, Q, bucket, rir, rir_gain, Hc,
                                                                  tw.get(e_for(M)));
}

void launch_spectrum(int logN, const DevBatch& B, const Queues& Q, const float* rir, const float* rir_gain,
                     float2* Hc, Twiddles tw, int grid, cudaStream_t st) {
    const int b = logN - kMinLog;
    switch (logN) {
        case 11: spectrum_m<1024>(B, Q, b, rir, rir_gain, Hc, tw, grid, st); break;
        case 12: spectrum_m<2048>(B, Q, b, rir, rir_gain, Hc, tw, grid, st); break;
        case 13: spectrum_m<4096>(B, Q, b, rir, rir_gain, Hc, tw, grid, st); break;
        case 14: spectrum_m<8192>(B, Q, b, rir, rir_gain, Hc, tw, grid, st); break;
        default: break;
    }
}

template <int M>
static void forward_m(const DevBatch& B, const Queues& Q, int bucket, const float* x,
                      const float* gains, const float2* Hc, float* y, float* tails,
                      Twiddles tw, int grid, cudaStream_t st) {
    k_forward<M><<<grid, FwdCfg<M>::T, smem_forward<M>(), st>>>(B, Q, bucket, x, gains, Hc, y, tails,
                                                                tw.get(FwdCfg<M>::E));
}

void launch_forward(int logN, const DevBatch& B, const Queues& Q, const float* x, const float* gains,
                    const float2* Hc, float* y, float* tails, Twiddles tw, int grid,
                    cudaStream_t st) {
    const int b = logN - kMinLog;
    switch (logN) {
        case 11: forward_m<1024>(B, Q, b, x, gains, Hc, y, tails, tw, grid, st); break;
        case 12: forward_m<2048>(B, Q, b, x, gains, Hc, y, tails, tw, grid, st); break;
        case 13: forward_m<4096>(B, Q, b, x, gains, Hc, y, tails, tw, grid, st); break;
        case 14: forward_m<8192>(B, Q, b, x, gains, Hc, y, tails, tw, grid, st); break;
        default: break;
    }
}

void launch_fixup(const DevBatch& B, float* y, const float* tails, cudaStream_t st) {
    int grid = B.NSEG < 4096 ? B.NSEG : 4096;
    if (grid < 1) grid = 1;
    k_fixup<<<dim3(grid, B.J > 0 ? B.J : 1), 256, 0, st>>>(B, y, tails);
}

int threads_for(int logN) { const int M = 1 << (logN - 1); return M / e_for(M); }

template <typename K>
static int occ(K kernel, int threads, int smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
    return n > 0 ? n : 1;
}

int occupancy_spectrum(int logN) {
    switch (logN) {
        case 11: return occ(k_spectrum<1024>, threads_for(11), smem_spectrum<1024>());
        case 12: return occ(k_spectrum<2048>, threads_for(12), smem_spectrum<2048>());
        case 13: return occ(k_spectrum<4096>, threads_for(13), smem_spectrum<4096>());
        case 14: return occ(k_spectrum<8192>, threads_for(14), smem_spectrum<8192>());
    }
    return 1;
}

int occupancy_forward(int logN) {
    switch (logN) {
        case 11: return occ(k_forward<1024>, FwdCfg<1024>::T, smem_forward<1024>());
        case 12: return occ(k_forward<2048>, FwdCfg<2048>::T, smem_forward<2048>());
        case 13: return occ(k_forward<4096>, FwdCfg<4096>::T, smem_forward<4096>());
        case 14: return occ(k_forward<8192>, FwdCfg<8192>::T, smem_forward<8192>());
    }
    return 1;
}

}  // namespace rsim
