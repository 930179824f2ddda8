// Backward path: the adjoint of the overlap-add filter-and-mix.
//
// With g_j = dLoss/dy_j (y over [0, Nx)), the adjoint of Eq. 2 is
//   dx_i[m]   = alpha_i sum_j sum_k hhat_ij[k] g_j[m + k]      (correlation)
//   dh_ij[k]  = alpha_i sum_n g_j[n] x_i[n - k],  k < L_ij     (0 beyond)
//   dalpha_i  = sum_j <g_j, hhat_ij * x_i> = <c_i, x_i>,  c_i = dx_i / alpha_i
// Block by block (hop = N - L_max + 1) with G_jb = rFFT_N(g_j[b hop, b hop + N)):
//   c_i on [b hop, (b+1) hop) = irFFT_N(sum_j conj(H_ij) G_jb)[0, hop)
//   dh_ij = alpha_i / N * irFFT(sum_b conj(X_ib) G_jb)[0, L_ij)
// Neither wraps around: lags and positions stay below hop + L_max - 1 = N.
#include "rsim_fft.cuh"
#include "rsim_internal.cuh"
#include "rsim_tmem.cuh"

namespace rsim {

__device__ __forceinline__ double block_sum_d(double v, double* sd) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sd[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < nw) ? sd[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

// ---------------------------------------------------------------------------
// K7: persistent over (backward segment, source) tiles
// ---------------------------------------------------------------------------
// Per block b of the segment, for source i:
//   X = rFFT_N(x_i block)                                  registers (pair layout)
//   for each mic j: G_j = rFFT_N(g_j[b hop, b hop + hop + L_max - 1))
//       C += conj(Hc_ij) G_j                               folded into the inverse
//                                                          pre-processing of the last mic
//       W_j += conj(X) G_j                                 registers, kept across
//                                                          the segment
//   c = irFFT_N(C)[0, hop): dx_i = alpha_i c, dalpha_i += <c, x_i> (computed
//   as sum_k C[k] conj(X[k]) on the spectra, by Parseval)
// and at the end of the segment dh partial_ij = irFFT_N(W_j)[0, L_ij).
// Every transform input (x block, g windows) is prefetched into one of NST
// shared-memory stages while the previous transform runs: with two stages by
// one bulk copy per block (the copy engine moves its whole 16-byte chunks and
// completes an mbarrier the readers wait on, with a bounded wait), with one
// stage by per-thread cp.async.  Transform exchanges alternate between NSM
// buffers (one barrier per exchange when NSM = 2).  The source's RIR spectra are staged once per
// tile; twiddles are copied to shared memory once per CTA.  Microphones go in
// groups of kJG (the source spectrum is recomputed per group; dx of later
// groups is added to the first group's).
template <int M>
struct BwdCfg {
    static constexpr int E = M == 4096 ? 16 : e_for(M);
    static constexpr int T = M / E;
    static constexpr int NSM = M <= 4096 ? 2 : 1;    // exchange buffers
    static constexpr int NST = M == 2048 ? 1 : 2;    // input stages
    static constexpr bool kStageH = M <= 4096;
    static constexpr bool kTwSmem = M <= 4096;
    static constexpr int kMinBlocks = M <= 2048 ? 2 : 1;
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t SM_LEN = a16(sizeof(float2) * padded_len(M));
    static constexpr size_t ST_LEN = sizeof(float) * (2 * M + 8);   // + room for the chunk offset
    static constexpr size_t o_sm = 0;
    static constexpr size_t o_st = o_sm + NSM * SM_LEN;
    static constexpr size_t o_hs = a16(o_st + NST * ST_LEN);
    static constexpr size_t o_tw = a16(o_hs + (kStageH ? sizeof(float2) * kJG * M : 0));
    static constexpr size_t bytes = a16(o_tw + (kTwSmem ? sizeof(float2) * FftPlan<M, E>::TW_LEN : 0));
};

static_assert(kJG == 2, "the backward tile loop is written for microphone pairs");

// MG: more microphones than one group (J > kJG): later groups add their dx to
// the first group's.  Without it dx is only written, which keeps the
// read-modify-write path out of the common kernel.
// CACHED: the forward kept every block's source spectrum (B.xspec): the source
// step of each microphone group stages it by one bulk copy instead of
// transforming the block.
template <int M, bool MG, bool CACHED>
__global__ void __launch_bounds__(BwdCfg<M>::T, BwdCfg<M>::kMinBlocks)
k_backward(DevBatch B, Queues Q, int bucket, const float* __restrict__ gy, const float* __restrict__ x,
           const float* __restrict__ gains, const float2* __restrict__ Hc, float* __restrict__ dx,
           float* __restrict__ dhp, float* __restrict__ dap, const float2* __restrict__ twg) {
    using L = BwdCfg<M>;
    constexpr int E = L::E;
    constexpr int T = L::T;
    constexpr int NST = L::NST;
    constexpr bool kBulk = NST == 2;      // inputs staged by bulk copies completing on mbarriers
    static_assert(!CACHED || kBulk, "the cached source spectra are staged by bulk copies");
    constexpr bool kPaired = PairedSplit<M, E>::ok;   // split in registers (paired layout)
    using Pl = FftPlan<M, E>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Exch<L::NSM> ex{reinterpret_cast<float2*>(smem_raw + L::o_sm),
                    reinterpret_cast<float2*>(smem_raw + L::o_sm + (L::NSM - 1) * L::SM_LEN), 0};
    float* st0 = reinterpret_cast<float*>(smem_raw + L::o_st);
    float2* hs = reinterpret_cast<float2*>(smem_raw + L::o_hs);
    __shared__ double sd[32];
    __shared__ __align__(8) uint64_t mbar[2];
    const int t = threadIdx.x;
    if constexpr (kBulk) {
        if (t == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
    uint32_t ph = 0;                             // bit b: parity of the next phase of stage b
    int off0 = 0, off1 = 0;                      // float offset of the data in stage 0 / 1
    bool bad = false;                            // a bounded wait ran out (no new copies then)
    const float2* tw = twg;
    if constexpr (L::kTwSmem) {
        float2* tws = reinterpret_cast<float2*>(smem_raw + L::o_tw);
        for (int k = t; k < Pl::TW_LEN; k += T) tws[k] = twg[k];
        __syncthreads();
        tw = tws;
    }
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    // first bin of this thread's pairs: t (pair layout) or its paired butterfly
    const int kt = kPaired ? paired_butterfly<T>(t) : t;
    int sc = 0;                                  // stage holding the next transform input
    auto stage = [&](int k) { return st0 + (NST == 2 ? k : 0) * (2 * M + 8); };
    bool stop = false;                           // a wait ran out: the remaining pieces are skipped
    for_each_piece(B, bucket, blockIdx.x, [&](int pc, int, int u, int i, int64_t b0, int64_t b1) {
        if (stop) return;
        const int64_t nx = B.n_x[u];
        const int64_t ny = B.n_y[u];
        const int hop = B.hop[u];
        const int lmax = B.Lmax[u];
        const int J = B.J;
        const int sb = B.src0[u], rb = B.rir0[u];
        const float a = __ldg(gains + sb + i);
        const float* xi = x + B.xoff[sb + i];
        float* dxi = dx ? dx + B.xoff[sb + i] : nullptr;
        float da = 0.f;              // <c, x_i> over the segment
        for (int j0 = 0; j0 < J; j0 += kJG) {
            const int jn = min(kJG, J - j0);
            // queue a real block into stage k (bulk copy + mbarrier, or cp.async)
            auto stage_in = [&](int k, const float* src, int64_t len) {
                if constexpr (kBulk) {
                    const int off = stage_real_bulk<M, E>(stage(k), src, len, &mbar[k], t, B.test_withhold != 0);
                    if (k) off1 = off; else off0 = off;
                } else {
                    stage_real_async<M, E>(stage(k), src, len, t);
                }
            };
            auto stage_x = [&](int k, int64_t b) {
                if constexpr (CACHED) {          // the forward's spectrum of the block (2M floats)
                    stage_in(k, reinterpret_cast<const float*>(reinterpret_cast<const char*>(B.xspec) +
                                                               B.xspec_off[sb + i]) + b * 2 * M,
                             2 * M);
                } else {
                    const int64_t p = b * hop;
                    stage_in(k, xi + p, min((int64_t)hop, nx - p));
                }
            };
            auto stage_g = [&](int k, int64_t b, int j) {
                const int64_t p = b * hop;
                stage_in(k, gy + B.yoff[u] + (int64_t)j * ny + p, min((int64_t)(hop + lmax - 1), ny - p));
            };
            // takes the staged input into v and queues the next one (if any) into the other stage
            auto next_input = [&](float2 (&v)[E], int64_t b, int nj) {
                if constexpr (kBulk) {
                    if (!bad && !mbar_wait_bounded(&mbar[sc], (ph >> sc) & 1u)) {
                        // give the copy one more bounded chance to land before the
                        // stage is abandoned, so none is left in flight at exit
                        mbar_wait_bounded(&mbar[sc], (ph >> sc) & 1u, 100000000ull);
                        bad = true;
                    }
                    ph ^= 1u << sc;
                    load_staged_at<M, E>(v, stage(sc), sc ? off1 : off0, t);
                } else {
                    cp_async_wait<0>();
                    __syncthreads();
                    load_staged_strided<M, E>(v, stage(sc), t);
                    __syncthreads();
                }
                if (kBulk && bad) {
                    // stop feeding the stages after a wait ran out
                } else if (nj >= 0) {
                    stage_g(sc ^ (NST - 1), b, nj);
                } else if (b + 1 < b1) {
                    stage_x(sc ^ (NST - 1), b + 1);
                }
                if constexpr (!kBulk) cp_async_commit();
                sc ^= (NST - 1);
            };
            // X of a block from the stage (pair k = (X[k], X[M - k])); queues microphone
            // j0's window, then a barrier: every thread is done with the stage before a
            // later step's copy refills it (a source step has no transform to provide one)
            auto take_x = [&](float2 (&Xo)[E], int64_t b) {
                if (!bad && !mbar_wait_bounded(&mbar[sc], (ph >> sc) & 1u)) {
                    mbar_wait_bounded(&mbar[sc], (ph >> sc) & 1u, 100000000ull);
                    bad = true;
                }
                ph ^= 1u << sc;
                const float4* s4 = reinterpret_cast<const float4*>(stage(sc));
#pragma unroll
                for (int q = 0; q < E / 2; ++q) {
                    const float4 e4 = s4[kt + q * T];
                    Xo[2 * q] = make_float2(e4.x, e4.y);
                    Xo[2 * q + 1] = make_float2(e4.z, e4.w);
                }
                if (!bad) stage_g(sc ^ 1, b, j0);
                sc ^= 1;
                __syncthreads();
            };
            float2 W[kJG][E];
#pragma unroll
            for (int jj = 0; jj < kJG; ++jj)
#pragma unroll
                for (int e = 0; e < E; ++e) W[jj][e] = make_float2(0.f, 0.f);
            __syncthreads();                     // stages and spectra are free
            if constexpr (L::kStageH) {
                for (int jj = 0; jj < jn; ++jj)
                    stage_spectrum_async<M, E>(hs + jj * M, Hc + (int64_t)(rb + i * J + j0 + jj) * B.MMAX, t);
            }
            stage_x(sc, b0);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            // C += conj(H_j) G_j and W_j += conj(X) G_j; G_j from the spectrum in z
            // (split here) or already split in registers (paired layout)
            auto mac = [&](float2 (&Wj)[E], float2 (&C)[E], const float2 (&X)[E], const float2* z,
                           const float2 (&G)[E], int jj) {
                const float2* Hg = Hc + (int64_t)(rb + i * J + j0 + jj) * B.MMAX;
#pragma unroll
                for (int q = 0; q < E / 2; ++q) {
                    const int k = kt + q * T;
                    float2 ga, gb;
                    if constexpr (kPaired) {
                        ga = G[2 * q];
                        gb = G[2 * q + 1];
                    } else {
                        split_pair<M>(z, wsplit, k, ga, gb);
                    }
                    const float4 hh = L::kStageH ? reinterpret_cast<const float4*>(hs + jj * M)[k]
                                                 : __ldg(reinterpret_cast<const float4*>(Hg) + k);
                    const float2 ha = make_float2(hh.x, hh.y), hb = make_float2(hh.z, hh.w);
                    if (k == 0) {            // slot 0 holds two real bins
                        C[0].x += ha.x * ga.x;
                        C[0].y += ha.y * ga.y;
                        Wj[0].x += X[0].x * ga.x;
                        Wj[0].y += X[0].y * ga.y;
                    } else {
                        C[2 * q] = cadd(C[2 * q], cmulc(ha, ga));
                        Wj[2 * q] = cadd(Wj[2 * q], cmulc(X[2 * q], ga));
                    }
                    C[2 * q + 1] = cadd(C[2 * q + 1], cmulc(hb, gb));
                    Wj[2 * q + 1] = cadd(Wj[2 * q + 1], cmulc(X[2 * q + 1], gb));
                }
            };
            for (int64_t b = b0; b < b1; ++b) {
                const int64_t pos = b * hop;
                const int64_t lim = nx - pos;
                float2 v[E], X[E], C[E];
#pragma unroll
                for (int e = 0; e < E; ++e) C[e] = make_float2(0.f, 0.f);
                // step 0 transforms the source block, step 1 + jj the window of mic j0 + jj;
                // one loop body (not unrolled) so the transform code is emitted once
#pragma unroll 1
                for (int sp = 0; sp <= kJG; ++sp) {
                    if (sp > jn) break;
                    if constexpr (CACHED) {
                        if (sp == 0) {
                            take_x(X, b);
                            continue;
                        }
                    }
                    next_input(v, b, sp < jn ? j0 + sp : -1);
                    if constexpr (kPaired) {
                        float2 G[E];
                        rfft_paired<M, E, false>(G, v, ex, tw, t, kt);
                        if (sp == 0) {
#pragma unroll
                            for (int e = 0; e < E; ++e) X[e] = G[e];
                        } else if (sp == 1) {
                            mac(W[0], C, X, nullptr, G, 0);
                        } else {
                            mac(W[1], C, X, nullptr, G, 1);
                        }
                    } else {
                        const float2* z = rfft_x<M, E, false>(v, ex, tw, t);
                        // X is kept while the next steps' transforms rewrite z (with one
                        // exchange buffer z is the same address at every step)
                        if (sp == 0) split_forward_now<M, E>(X, z, wsplit, t);
                        else if (sp == 1) mac(W[0], C, X, z, v, 0);
                        else mac(W[1], C, X, z, v, 1);
                    }
                }
                // <c, x_block> by Parseval on the half spectra already in registers
                // (x_block is zero beyond its length, so only n < hop counts):
                // sum_n c x = sum_k C[k] conj(X[k]) over all N bins, i.e. bins 0
                // and N/2 once and every other bin of the half spectrum twice.
#pragma unroll
                for (int q = 0; q < E / 2; ++q) {
                    const int k = kt + q * T;
                    const float p0 = C[2 * q].x * X[2 * q].x + C[2 * q].y * X[2 * q].y;
                    const float p1 = C[2 * q + 1].x * X[2 * q + 1].x + C[2 * q + 1].y * X[2 * q + 1].y;
                    da += (k == 0 ? p0 : 2.f * p0) + 2.f * p1;
                }
                if constexpr (kPaired) irfft_paired<M, E>(v, C, ex, tw, t, kt);
                else irfft_x<M, E, false>(v, C, ex, tw, t);
                if (dxi) {
                    // samples [0, min(hop, Nx - pos)) of the block; the first mic group
                    // writes, later groups add; pairs go out as one 8-byte store when aligned
                    float* dst = dxi + pos;
                    const int ilim = (int)min((int64_t)hop, lim);
                    const bool pairs = ((reinterpret_cast<uintptr_t>(dst) & 7) == 0) && j0 == 0;
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
                        const float d0 = a * v[q].x, d1 = a * v[q].y;
                        if (pairs && n + 1 < ilim) {
                            if (RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B)))
                                *reinterpret_cast<float2*>(dst + n) = make_float2(d0, d1);
                        } else if constexpr (MG) {
                            if (n < ilim && RSIM_STORE_OK(B, dst + n, dx, RSIM_X_BYTES(B)))
                                dst[n] = (j0 == 0) ? d0 : dst[n] + d0;
                            if (n + 1 < ilim && RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B)))
                                dst[n + 1] = (j0 == 0) ? d1 : dst[n + 1] + d1;
                        } else {
                            if (n < ilim && RSIM_STORE_OK(B, dst + n, dx, RSIM_X_BYTES(B))) dst[n] = d0;
                            if (n + 1 < ilim && RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B))) dst[n + 1] = d1;
                        }
                    }
                }
            }
            // dh partials of this segment for mics j0 .. j0 + jn - 1 (one loop body)
#pragma unroll 1
            for (int jj = 0; jj < jn; ++jj) {
                float2 v[E], Pw[E];
#pragma unroll
                for (int e = 0; e < E; ++e) Pw[e] = jj ? W[1][e] : W[0][e];
                if constexpr (kPaired) irfft_paired<M, E>(v, Pw, ex, tw, t, kt);
                else irfft_x<M, E, false>(v, Pw, ex, tw, t);
                const int r = rb + i * J + j0 + jj;
                const int Lr = B.L[r];
                float* out = dhp + B.piece_dh[pc] + (B.lpre[r] - B.lpre[rb + i * J]);
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const int n = 2 * (t + q * T);
                    if (n < Lr && RSIM_STORE_OK(B, out + n, dhp, B.NDHP * 4)) out[n] = v[q].x;
                    if (n + 1 < Lr && RSIM_STORE_OK(B, out + n + 1, dhp, B.NDHP * 4)) out[n + 1] = v[q].y;
                }
            }
        }
        const double tot = block_sum_d((double)da, sd);
        if (t == 0) dap[(int64_t)pc * kMaxSources] = (float)tot;
        if constexpr (kBulk) {
            if (__syncthreads_or(bad)) {         // a copy never completed: report and stop
                if (t == 0) atomicOr(B.err, kErrWaitTimeout);
                stop = true;
            }
        }
    });
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// K7 (N <= 8192): persistent over (block run, source group) tiles, RIR-gradient
// accumulators in TMEM
// ---------------------------------------------------------------------------
// A tile is a run of consecutive blocks [b0, b1) of one utterance (chosen by
// the planner so that tiles cost about the same) and up to IG of its sources.
// Per block b and microphone group j0 .. j0 + jn - 1:
//   G_j = rFFT_N(g_j[b hop, b hop + N))          once per microphone, registers
//   for each source i of the tile:
//     X_i = rFFT_N(x_i block)                     once per source
//     W_ij += conj(X_i) G_j                       accumulators in TMEM
//     C_i = sum_j conj(Hc_ij) G_j                 RIR spectra from L2
//     dalpha_i += <c_i, x_i block> = sum_k C_i conj(X_i) (Parseval)
//     dx_i block = alpha_i irFFT_N(C_i)[0, hop)  (added to earlier groups')
// and at the end of the run dh partial_ij = irFFT_N(W_ij)[0, L_ij).  That is
// 2I + J transforms per block, the method's minimum (a per-source tile
// recomputes every G_j per source: I (J + 2)).  The I x jn accumulators of a
// tile do not fit in registers: each is a half spectrum spread over the CTA
// like the transforms (2E floats per thread), held in TMEM columns of the
// thread's own lane and read and written once per block with tcgen05.ld/st.
// Transform inputs are staged as in the per-source kernel: one bulk copy per
// input into one of two shared-memory stages, completing on an mbarrier with
// a bounded wait, issued while the previous transform runs; exchanges
// alternate between two buffers (one barrier each).
template <int M>
struct BwdTmCfg {
    static constexpr int E = M == 4096 ? 16 : e_for(M);
    static constexpr int T = M / E;
    static constexpr int kMinBlocks = M <= 2048 ? 2 : 1;
    static constexpr int kWCols = 2 * E * (T / 128);          // TMEM columns per accumulator
    static constexpr int kCols = kMinBlocks == 2 ? 256 : 512;  // TMEM columns per CTA
    static constexpr int IG = kCols / (kWCols * kJG);          // sources per tile
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t SM_LEN = a16(sizeof(float2) * padded_len(M));
    static constexpr size_t ST_LEN = sizeof(float) * (2 * M + 8);   // + room for the chunk offset
    static constexpr size_t o_sm = 0;
    static constexpr size_t o_st = o_sm + 2 * SM_LEN;
    static constexpr size_t o_tw = a16(o_st + 2 * ST_LEN);
    // the current source's RIR spectra (one microphone group), staged by bulk copies
    // issued before its forward transform: where one CTA per SM leaves the room
    static constexpr bool kStageH = kMinBlocks == 1;
    static constexpr size_t o_hs = a16(o_tw + sizeof(float2) * FftPlan<M, E>::TW_LEN);
    static constexpr size_t bytes = a16(o_hs + (kStageH ? sizeof(float2) * kJG * M : 0));
    static_assert(T % 128 == 0, "every TMEM lane quadrant holds whole runs of columns");
    static_assert(bytes <= 227 * 1024 - 1024, "shared memory of one CTA");
    static_assert(IG >= 1 && IG <= kMaxSources, "source group");
};

// CACHED: the forward kept every block's source spectrum (B.xspec), which source steps read
// instead of transforming the block
template <int M, bool MG, bool CACHED>
__global__ void __launch_bounds__(BwdTmCfg<M>::T, BwdTmCfg<M>::kMinBlocks)
k_backward_tm(DevBatch B, Queues Q, int bucket, const float* __restrict__ gy, const float* __restrict__ x,
              const float* __restrict__ gains, const float2* __restrict__ Hc, float* __restrict__ dx,
              float* __restrict__ dhp, float* __restrict__ dap, const float2* __restrict__ twg) {
    using L = BwdTmCfg<M>;
    constexpr int E = L::E;
    constexpr int T = L::T;
    constexpr int IG = L::IG;
    constexpr bool kPaired = PairedSplit<M, E>::ok;   // split in registers (paired layout)
    static_assert(IG == bwd_src_group(ilog2(M) + 1), "the planner's source groups");
    using Pl = FftPlan<M, E>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Exch<2> ex{reinterpret_cast<float2*>(smem_raw + L::o_sm),
               reinterpret_cast<float2*>(smem_raw + L::o_sm + L::SM_LEN), 0};
    float* st0 = reinterpret_cast<float*>(smem_raw + L::o_st);
    float2* hs = reinterpret_cast<float2*>(smem_raw + L::o_hs);
    __shared__ double sd[32];
    __shared__ __align__(8) uint64_t mbar[3];      // two input stages, the RIR spectra
    __shared__ uint32_t tmem_base;
    // the piece's per-source gains and offsets and its utterance's output offset, read once
    // per piece (every step reads them: from global memory each read would sit on the step's path)
    __shared__ float s_gain[IG];
    __shared__ int64_t s_xoff[IG], s_xso[IG];
    __shared__ int64_t s_yoff;
    const int t = threadIdx.x;
    if (chunk_empty(B, bucket, blockIdx.x)) return;   // before any TMEM is taken
    if (t < 32) {                                // warp 0 takes the CTA's TMEM columns
        tmem_alloc(&tmem_base, L::kCols);
        tmem_relinquish();
    }
    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        mbar_init_fence();
    }
    float2* tws = reinterpret_cast<float2*>(smem_raw + L::o_tw);
    for (int k = t; k < Pl::TW_LEN; k += T) tws[k] = twg[k];
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const float2* tw = tws;
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    // accumulator s of this thread: columns s * kWCols + (its run) of its lane
    const uint32_t tacc = tmem_thread_addr<E>(tmem_base, t);
    auto wslot = [&](int s) { return tacc + (uint32_t)(s * L::kWCols); };
    uint32_t ph = 0;                             // bit b: parity of the next phase of barrier b
    int off0 = 0, off1 = 0;                      // float offset of the data in stage 0 / 1
    bool bad = false;                            // a bounded wait ran out (no new copies then)
    // first bin of this thread's pairs: t (pair layout) or its paired butterfly
    const int kt = kPaired ? paired_butterfly<T>(t) : t;
    int sc = 0;                                  // stage holding the next transform input
    auto stage = [&](int k) { return st0 + k * (2 * M + 8); };
    // waits (bounded) for barrier b's current phase; a wait that runs out marks the
    // CTA bad after one more bounded chance for the copy to land
    auto wait_bar = [&](int b) {
        if (!bad && !mbar_wait_bounded(&mbar[b], (ph >> b) & 1u)) {
            mbar_wait_bounded(&mbar[b], (ph >> b) & 1u, 100000000ull);
            bad = true;
        }
        ph ^= 1u << b;
    };
    bool h_pending = false;                      // a spectrum copy was issued and not yet waited for
    // the forward kept every block's source spectrum: a source step stages it instead of
    // the block and needs no forward transform
    constexpr bool cached = CACHED;
    bool stop = false;                           // a wait ran out: the remaining pieces are skipped
    for_each_piece(B, bucket, blockIdx.x, [&](int pc, int, int u, int i0, int64_t b0, int64_t b1) {
        if (stop) return;
        const int64_t nx = B.n_x[u];
        const int64_t ny = B.n_y[u];
        const int hop = B.hop[u];
        const int lmax = B.Lmax[u];
        const int J = B.J;
        const int I = min(IG, B.n_src[u] - i0);
        const int sb = B.src0[u] + i0, rb = B.rir0[u];
        __syncthreads();                         // the previous piece's readers are done
        if (t < I) {
            s_gain[t] = __ldg(gains + sb + t);
            s_xoff[t] = B.xoff[sb + t];
            s_xso[t] = cached ? B.xspec_off[sb + t] : 0;
        }
        if (t == 0) s_yoff = B.yoff[u];          // (read after the group's first barrier)
        float da[IG];                            // <c_i, x_i> over the run, per source
#pragma unroll
        for (int q = 0; q < IG; ++q) da[q] = 0.f;
        for (int j0 = 0; j0 < J; j0 += kJG) {
            const int jn = min(kJG, J - j0);
            const int nsteps = jn + I;           // transforms per block: the G_j, then the X_i
            // queue the input of step k of block b into stage kk
            auto stage_step = [&](int kk, int64_t b, int k) {
                const int64_t p = b * hop;
                const float* src;
                int64_t len;
                if (k < jn) {
                    src = gy + s_yoff + (int64_t)(j0 + k) * ny + p;
                    len = min((int64_t)(hop + lmax - 1), ny - p);
                } else if (cached) {             // the forward's spectrum of the block
                    src = reinterpret_cast<const float*>(reinterpret_cast<const char*>(B.xspec) +
                                                         s_xso[k - jn]) + b * 2 * M;
                    len = 2 * M;
                } else {
                    src = x + s_xoff[k - jn] + p;
                    len = min((int64_t)hop, nx - p);
                }
                const int off = stage_real_bulk<M, E>(stage(kk), src, len, &mbar[kk], t, B.test_withhold != 0);
                if (kk) off1 = off; else off0 = off;
            };
            // takes the staged input of step k into v and queues the next step's
            auto next_input = [&](float2 (&v)[E], int64_t b, int k) {
                wait_bar(sc);
                load_staged_at<M, E>(v, stage(sc), sc ? off1 : off0, t);
                if (!bad) {
                    if (k + 1 < nsteps) stage_step(sc ^ 1, b, k + 1);
                    else if (b + 1 < b1) stage_step(sc ^ 1, b + 1, 0);
                }
                sc ^= 1;
            };
            // when step k is a source step its RIR spectra move into hs, once the readers of
            // hs are done: without the cache at the start of step k (the previous source
            // step's spectral products passed the barriers of its inverse transform; the
            // copy lands while this step's forward transform runs), with it as early as the
            // previous step allows (after its spectral products and a barrier, or at the
            // end of a microphone step)
            auto stage_h = [&](int k) {
                if constexpr (L::kStageH) {
                    if (k < jn || k >= nsteps || bad) return;
                    h_pending = true;
                    if (t == 0) {
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(&mbar[2], (uint32_t)(jn * M * sizeof(float2)));
                        for (int jj = 0; jj < jn; ++jj)
                            bulk_copy_g2s(hs + jj * M, Hc + (int64_t)(rb + (i0 + k - jn) * J + j0 + jj) * B.MMAX,
                                          (uint32_t)(M * sizeof(float2)), &mbar[2]);
                    }
                }
            };
            // zero this group's accumulators (no other thread reads this thread's columns)
            {
                float2 z[E];
#pragma unroll
                for (int e = 0; e < E; ++e) z[e] = make_float2(0.f, 0.f);
                for (int s2 = 0; s2 < I * kJG; ++s2) tmem_store<E>(wslot(s2), z);
            }
            __syncthreads();                     // stages are free
            stage_step(sc, b0, 0);
            // the stage's ragged ends and zero fill are plain stores by every thread:
            // visible to all readers after this barrier (later inputs are staged a whole
            // transform, barriers included, before they are read)
            __syncthreads();
            for (int64_t b = b0; b < b1; ++b) {
                const int64_t pos = b * hop;
                float2 G[kJG][E];
                // a source step's work before its inverse transform: W_ij += conj(X_i) G_j
                // (TMEM), C = sum_j conj(H_ij) G_j, and <c, x_block> by Parseval
                auto src_pre = [&](int k, int i, const float2 (&Z)[E], float2 (&C)[E]) {
#pragma unroll 1
                    for (int jj = 0; jj < jn; ++jj) {
                        float2 Wv[E];
                        tmem_load<E>(Wv, wslot(i * kJG + jj));
#pragma unroll
                        for (int q = 0; q < E / 2; ++q) {
                            const float2 ga = jj ? G[1][2 * q] : G[0][2 * q];
                            const float2 gb = jj ? G[1][2 * q + 1] : G[0][2 * q + 1];
                            if (kt + q * T == 0) {   // slot 0 holds two real bins
                                Wv[0].x += Z[0].x * ga.x;
                                Wv[0].y += Z[0].y * ga.y;
                            } else {
                                Wv[2 * q] = cadd(Wv[2 * q], cmulc(Z[2 * q], ga));
                            }
                            Wv[2 * q + 1] = cadd(Wv[2 * q + 1], cmulc(Z[2 * q + 1], gb));
                        }
                        tmem_store<E>(wslot(i * kJG + jj), Wv);
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e) C[e] = make_float2(0.f, 0.f);
                    if constexpr (L::kStageH) {
                        if (h_pending && bad) {
                            // a stage wait ran out after this copy was issued: still let it land
                            mbar_wait_bounded(&mbar[2], (ph >> 2) & 1u, 100000000ull);
                            ph ^= 1u << 2;
                        } else if (h_pending) {
                            wait_bar(2);
                        }
                        h_pending = false;
                    }
#pragma unroll
                    for (int jj = 0; jj < kJG; ++jj) {
                        if (jj >= jn) break;
                        const float4* Hg = L::kStageH ? reinterpret_cast<const float4*>(hs + jj * M)
                                                      : reinterpret_cast<const float4*>(
                                                            Hc + (int64_t)(rb + (i0 + i) * J + j0 + jj) * B.MMAX);
#pragma unroll
                        for (int q = 0; q < E / 2; ++q) {
                            const int kb = kt + q * T;
                            const float4 hh = L::kStageH ? Hg[kb] : __ldg(Hg + kb);
                            const float2 ha = make_float2(hh.x, hh.y), hb = make_float2(hh.z, hh.w);
                            const float2 ga = jj ? G[1][2 * q] : G[0][2 * q];
                            const float2 gb = jj ? G[1][2 * q + 1] : G[0][2 * q + 1];
                            if (kb == 0) {
                                C[0].x += ha.x * ga.x;
                                C[0].y += ha.y * ga.y;
                            } else {
                                C[2 * q] = cadd(C[2 * q], cmulc(ha, ga));
                            }
                            C[2 * q + 1] = cadd(C[2 * q + 1], cmulc(hb, gb));
                        }
                    }
                    if constexpr (L::kStageH) {
                        // every thread is done with hs: the next source's spectra may come
                        // in while this step's inverse transform and stores run
                        if (cached && k + 1 < nsteps) {
                            __syncthreads();
                            stage_h(k + 1);
                        }
                    }
                    // <c, x_block> by Parseval on the half spectra (x_block is zero
                    // beyond its length): bins 0 and N/2 once, every other bin twice
                    float p = 0.f;
#pragma unroll
                    for (int q = 0; q < E / 2; ++q) {
                        const int kb = kt + q * T;
                        const float p0 = C[2 * q].x * Z[2 * q].x + C[2 * q].y * Z[2 * q].y;
                        const float p1 = C[2 * q + 1].x * Z[2 * q + 1].x + C[2 * q + 1].y * Z[2 * q + 1].y;
                        p += (kb == 0 ? p0 : 2.f * p0) + 2.f * p1;
                    }
#pragma unroll
                    for (int q = 0; q < IG; ++q) da[q] += (q == i) ? p : 0.f;
                };
                // dx = alpha c on samples [0, min(hop, Nx - pos)) of the block; the first
                // microphone group writes, later groups add; pairs go out as one 8-byte store
                auto dx_store = [&](int i, const float2 (&v)[E]) {
                    if (!dx) return;
                    const float a = s_gain[i];
                    float* dst = dx + s_xoff[i] + pos;
                    const int ilim = (int)min((int64_t)hop, nx - pos);
                    const bool pairs = ((reinterpret_cast<uintptr_t>(dst) & 7) == 0) && j0 == 0;
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
                        const float d0 = a * v[q].x, d1 = a * v[q].y;
                        if (pairs && n + 1 < ilim) {
                            if (RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B)))
                                *reinterpret_cast<float2*>(dst + n) = make_float2(d0, d1);
                        } else if constexpr (MG) {
                            if (n < ilim && RSIM_STORE_OK(B, dst + n, dx, RSIM_X_BYTES(B)))
                                dst[n] = (j0 == 0) ? d0 : dst[n] + d0;
                            if (n + 1 < ilim && RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B)))
                                dst[n + 1] = (j0 == 0) ? d1 : dst[n + 1] + d1;
                        } else {
                            if (n < ilim && RSIM_STORE_OK(B, dst + n, dx, RSIM_X_BYTES(B))) dst[n] = d0;
                            if (n + 1 < ilim && RSIM_STORE_OK(B, dst + n + 1, dx, RSIM_X_BYTES(B))) dst[n + 1] = d1;
                        }
                    }
                };
                auto keep_g = [&](int k, const float2 (&Z)[E]) {
                    if (k == 0) {
#pragma unroll
                        for (int e = 0; e < E; ++e) G[0][e] = Z[e];
                    } else {
#pragma unroll
                        for (int e = 0; e < E; ++e) G[1][e] = Z[e];
                    }
                };
                // X_i of a source step from the stage (pair kb = (X[kb], X[M - kb]))
                auto take_x = [&](float2 (&Z)[E], int k) {
                    wait_bar(sc);
                    const float4* sp = reinterpret_cast<const float4*>(stage(sc));
#pragma unroll
                    for (int q = 0; q < E / 2; ++q) {
                        const float4 e4 = sp[kt + q * T];
                        Z[2 * q] = make_float2(e4.x, e4.y);
                        Z[2 * q + 1] = make_float2(e4.z, e4.w);
                    }
                    if (!bad) {
                        if (k + 1 < nsteps) stage_step(sc ^ 1, b, k + 1);
                        else if (b + 1 < b1) stage_step(sc ^ 1, b + 1, 0);
                    }
                    sc ^= 1;
                };
                if constexpr (cached && kPaired) {
                    // one transform per step, at one place: a microphone step's forward
                    // (passes from butterfly t to butterfly kt, then the real split), a source
                    // step's inverse (the unsplit of C, passes from kt to t, conjugate) --
                    // the pass code is emitted once
#pragma unroll 1
                    for (int k = 0; k < nsteps; ++k) {
                        const bool src = k >= jn;
                        float2 v[E];
                        if (src) {
                            float2 Z[E], C[E];
                            take_x(Z, k);
                            src_pre(k, k - jn, Z, C);
                            paired_unsplit<M, E>(v, C, tw, kt);
                        } else {
                            next_input(v, b, k);
                        }
                        fft_passes_sel<M, E, 0, 2>(v, ex, tw, t, src ? kt : t, src ? t : kt);
                        if (!src) {
                            float2 Z[E];
                            paired_split<M, E>(Z, v, tw, kt);
                            keep_g(k, Z);
                            stage_h(k + 1);
                            continue;
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e) v[e] = conjf2(v[e]);
                        dx_store(k - jn, v);
                    }
                } else {
                    // one loop body for every step of the block (the transform code is
                    // emitted once per kind)
#pragma unroll 1
                    for (int k = 0; k < nsteps; ++k) {
                        float2 v[E], Z[E];
                        if constexpr (!cached) {
                            if (k >= jn) stage_h(k);
                        }
                        if (cached && k >= jn) {
                            take_x(Z, k);
                        } else {
                            next_input(v, b, k);
                            if constexpr (kPaired) {
                                rfft_paired<M, E, false>(Z, v, ex, tw, t, kt);
                            } else {
                                const float2* z = rfft_x<M, E, false>(v, ex, tw, t);
                                split_forward<M, E>(Z, z, wsplit, t);
                            }
                        }
                        if (k < jn) {
                            keep_g(k, Z);
                            if (cached) stage_h(k + 1);
                            continue;
                        }
                        const int i = k - jn;        // source of the tile; Z holds X_i
                        float2 C[E];
                        src_pre(k, i, Z, C);
                        if constexpr (kPaired) irfft_paired<M, E>(v, C, ex, tw, t, kt);
                        else irfft_x<M, E, false>(v, C, ex, tw, t);
                        dx_store(i, v);
                    }
                }
            }
            // dh partials of this run for the tile's sources and this microphone group
#pragma unroll 1
            for (int s2 = 0; s2 < I * jn; ++s2) {
                const int i = s2 / jn, jj = s2 - i * jn;
                float2 v[E], Wv[E];
                tmem_load<E>(Wv, wslot(i * kJG + jj));
                if constexpr (kPaired) irfft_paired<M, E>(v, Wv, ex, tw, t, kt);
                else irfft_x<M, E, false>(v, Wv, ex, tw, t);
                const int r = rb + (i0 + i) * J + j0 + jj;
                const int Lr = B.L[r];
                float* out = dhp + B.piece_dh[pc] + (B.lpre[r] - B.lpre[rb + i0 * J]);
#pragma unroll
                for (int q = 0; q < E; ++q) {
                    const int n = 2 * (t + q * T);
                    if (n < Lr && RSIM_STORE_OK(B, out + n, dhp, B.NDHP * 4)) out[n] = v[q].x;
                    if (n + 1 < Lr && RSIM_STORE_OK(B, out + n + 1, dhp, B.NDHP * 4)) out[n + 1] = v[q].y;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < IG; ++q) {
            if (q >= I) break;
            const double tot = block_sum_d((double)da[q], sd);
            if (t == 0) dap[(int64_t)pc * kMaxSources + q] = (float)tot;
        }
        if (__syncthreads_or(bad)) {             // a copy never completed: report and stop
            if (t == 0) atomicOr(B.err, kErrWaitTimeout);
            stop = true;
        }
    });
    // every thread's TMEM accesses are complete (each store waited); order them
    // before warp 0 frees the columns
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (t < 32) tmem_dealloc(tmem_base, L::kCols);
}

// ---------------------------------------------------------------------------
// K8: deterministic reduction of the per-segment partials
// ---------------------------------------------------------------------------
// grad_rir[r][k] = alpha_i / N * sum_pieces partial[k] for k < L_r, 0 for
// L_r <= k < Nh; grad_gains[s] = sum_pieces dalpha partial.  The pieces of
// the stream holding source i (s_first .. s_last, consecutive blocks of the
// utterance) are added in order.  With per-(i, j) gains (rir_gain non-NULL)
// the spectra already carry alpha_ij, the partials are the plain correlations
// c_r = corr(g_j, x_i) (times N), so grad_rir[r] = alpha_ij / N c_r and
// grad_gains[r] = <hhat_r, c_r> / N.
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads)
k_finalize(DevBatch B, const float* __restrict__ gains, const float* __restrict__ rir_gain,
           const float* __restrict__ rir, const float* __restrict__ dhp, const float* __restrict__ dap,
           float* __restrict__ grad_rir, float* __restrict__ grad_gains) {
    __shared__ float red[kFinThreads / 32];
    for (int r = blockIdx.x; r < B.R; r += gridDim.x) {
        const int u = B.rir_utt[r];
        const int i = (r - B.rir0[u]) / B.J;
        const int Lr = B.L[r], nh = B.rir_len[r];
        float* out = grad_rir + B.roff[r];
        if (B.logN[u] == 0) {
            for (int k = threadIdx.x; k < nh; k += blockDim.x)
                if (RSIM_STORE_OK(B, out + k, grad_rir, RSIM_RIR_BYTES(B))) out[k] = 0.f;
            if (rir_gain && grad_gains && threadIdx.x == 0 && RSIM_STORE_OK(B, grad_gains + r, grad_gains, 4 * B.R))
                grad_gains[r] = 0.f;
            continue;
        }
        const float inv_n = 1.f / (float)(1 << B.logN[u]);
        const float scale = (rir_gain ? rir_gain[r] : gains[B.src0[u] + i]) * inv_n;
        const float* h = rir_gain ? rir + B.roff[r] : nullptr;
        float dot = 0.f;                       // <hhat_r, c_r> (per-(i, j) gains)
        // the stream of source i: its first source, and the offset of RIR r in its partials
        const int sg = bwd_src_group(B.logN[u]);
        const int i0 = i / sg * sg;
        const int sidx = B.src0[u] + i0;
        const int64_t local = B.lpre[r] - B.lpre[B.rir0[u] + i0 * B.J];
        const int p0 = B.s_first[sidx], p1 = B.s_last[sidx];
        constexpr int kFinU = 4;               // taps per thread in flight (more cost occupancy)
        float acc[kFinU];
        // taps of this thread: k = threadIdx.x + c * blockDim.x
        const int ntap_passes = (nh + kFinThreads - 1) / kFinThreads;
        for (int c0 = 0; c0 < ntap_passes; c0 += kFinU) {
#pragma unroll
            for (int c = 0; c < kFinU; ++c) acc[c] = 0.f;
            for (int q = p0; q <= p1; ++q) {
                const float* src = dhp + B.piece_dh[q] + local;
#pragma unroll
                for (int c = 0; c < kFinU; ++c) {
                    const int k = threadIdx.x + (c0 + c) * kFinThreads;
                    if (k < Lr) acc[c] += src[k];
                }
            }
#pragma unroll
            for (int c = 0; c < kFinU; ++c) {
                const int k = threadIdx.x + (c0 + c) * kFinThreads;
                if (k < nh && RSIM_STORE_OK(B, out + k, grad_rir, RSIM_RIR_BYTES(B))) out[k] = k < Lr ? scale * acc[c] : 0.f;
                if (h && k < Lr) dot = fmaf(h[k], acc[c], dot);
            }
        }
        if (rir_gain && grad_gains) {          // block sum of dot, fixed order
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dot;
            __syncthreads();
            if (threadIdx.x == 0) {
                float s = 0.f;
                for (int w = 0; w < kFinThreads / 32; ++w) s += red[w];
                if (RSIM_STORE_OK(B, grad_gains + r, grad_gains, 4 * B.R)) grad_gains[r] = s * inv_n;
            }
            __syncthreads();
        }
    }
    if (grad_gains && !rir_gain) {
        for (int sidx = blockIdx.x * blockDim.x + threadIdx.x; sidx < B.S; sidx += gridDim.x * blockDim.x) {
            const int u = B.src_utt[sidx], i = sidx - B.src0[u];
            float acc = 0.f;
            if (B.logN[u] != 0) {
                const int sg = bwd_src_group(B.logN[u]);
                const int i0 = i / sg * sg;
                const int st = B.src0[u] + i0;
                for (int q = B.s_first[st]; q <= B.s_last[st]; ++q) acc += dap[(int64_t)q * kMaxSources + i - i0];
            }
            if (RSIM_STORE_OK(B, grad_gains + sidx, grad_gains, 4 * B.S)) grad_gains[sidx] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int M>
constexpr int smem_backward() { return (int)BwdCfg<M>::bytes; }
template <int M>
constexpr int smem_backward_tm() { return (int)BwdTmCfg<M>::bytes; }

// N <= 8192: the TMEM-accumulator kernel over (block run, source group) tiles;
// N = 16384: the per-source kernel (three spectra per thread at 16 values per
// thread would not fit its 128 registers)
template <int M>
static void backward_m(const DevBatch& B, const Queues& Q, int bucket, const float* g, const float* x,
                       const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                       Twiddles tw, int grid, cudaStream_t st) {
    if constexpr (M <= 4096) {
        auto kern = B.xspec ? (B.J > kJG ? k_backward_tm<M, true, true> : k_backward_tm<M, false, true>)
                            : (B.J > kJG ? k_backward_tm<M, true, false> : k_backward_tm<M, false, false>);
        kern<<<grid, BwdTmCfg<M>::T, smem_backward_tm<M>(), st>>>(B, Q, bucket, g, x, gains, Hc, dx, dhp,
                                                                  dap, tw.get(BwdTmCfg<M>::E));
    } else {
        auto kern = B.xspec ? (B.J > kJG ? k_backward<M, true, true> : k_backward<M, false, true>)
                            : (B.J > kJG ? k_backward<M, true, false> : k_backward<M, false, false>);
        kern<<<grid, BwdCfg<M>::T, smem_backward<M>(), st>>>(B, Q, bucket, g, x, gains, Hc, dx, dhp,
                                                                      dap, tw.get(BwdCfg<M>::E));
    }
}

void launch_backward(int logN, const DevBatch& B, const Queues& Q, const float* g, const float* x,
                     const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                     Twiddles tw, int grid, cudaStream_t st) {
    const int b = logN - kMinLog;
    switch (logN) {
        case 11: backward_m<1024>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, tw, grid, st); break;
        case 12: backward_m<2048>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, tw, grid, st); break;
        case 13: backward_m<4096>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, tw, grid, st); break;
        case 14: backward_m<8192>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, tw, grid, st); break;
        default: break;
    }
}

int bwd_threads(int logN) {
    switch (logN) {
        case 11: return BwdTmCfg<1024>::T;
        case 12: return BwdTmCfg<2048>::T;
        case 13: return BwdTmCfg<4096>::T;
        case 14: return BwdCfg<8192>::T;
    }
    return 1;
}

void launch_finalize(const DevBatch& B, const float* gains, const float* rir_gain, const float* rir,
                     const float* dhp, const float* dap,
                     float* grad_rir, float* grad_gains, cudaStream_t st) {
    int grid = B.R < 4096 ? B.R : 4096;
    if (grid < 1) grid = 1;
    k_finalize<<<grid, kFinThreads, 0, st>>>(B, gains, rir_gain, rir, dhp, dap, grad_rir, grad_gains);
}

template <typename K>
static int occ_b(K kernel, int threads, int smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
    return n > 0 ? n : 1;
}

// both microphone-group variants share the launch shape; the smaller occupancy rules
template <int M>
static int occ_bb() {
    int o = occ_b(k_backward<M, false, false>, BwdCfg<M>::T, smem_backward<M>());
    o = std::min(o, occ_b(k_backward<M, true, false>, BwdCfg<M>::T, smem_backward<M>()));
    if constexpr (BwdCfg<M>::NST == 2) {
        o = std::min(o, occ_b(k_backward<M, false, true>, BwdCfg<M>::T, smem_backward<M>()));
        o = std::min(o, occ_b(k_backward<M, true, true>, BwdCfg<M>::T, smem_backward<M>()));
    }
    return o;
}
// the TMEM kernels: also no more CTAs per SM than the SM's 512 TMEM columns hold
// (a CTA beyond that would wait in its allocation until another one exits)
template <int M>
static int occ_tm() {
    int n = 512 / BwdTmCfg<M>::kCols;
    const int o[4] = {occ_b(k_backward_tm<M, false, false>, BwdTmCfg<M>::T, smem_backward_tm<M>()),
                      occ_b(k_backward_tm<M, true, false>, BwdTmCfg<M>::T, smem_backward_tm<M>()),
                      occ_b(k_backward_tm<M, false, true>, BwdTmCfg<M>::T, smem_backward_tm<M>()),
                      occ_b(k_backward_tm<M, true, true>, BwdTmCfg<M>::T, smem_backward_tm<M>())};
    for (int k = 0; k < 4; ++k) n = o[k] < n ? o[k] : n;
    return n;
}

int occupancy_backward(int logN) {
    switch (logN) {
        case 11: return occ_tm<1024>();
        case 12: return occ_tm<2048>();
        case 13: return occ_tm<4096>();
        case 14: return occ_bb<8192>();
    }
    return 1;
}

}  // namespace rsim
