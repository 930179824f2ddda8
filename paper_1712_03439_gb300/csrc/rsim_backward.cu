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

namespace rsim {

__device__ __forceinline__ int pop_job_b(const Queues& Q, int kind, int b, int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int i = atomicAdd(&Q.next[Q.idx(kind, b)], 1);
        *slot = (i < Q.count[Q.idx(kind, b)]) ? Q.lst(kind, b)[i] : -1;
    }
    __syncthreads();
    return *slot;
}

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
// K7: persistent over backward segments (all sources of a segment per tile)
// ---------------------------------------------------------------------------
// Phase 1, per block b of the segment and mic j:
//   G_jb = rFFT_N(g_j[b hop, b hop + hop + L_max - 1))    stored once in this
//                                                          CTA's slice of Gc
// Phase 2, per source i (W_j in registers for the whole segment):
//   per block b:  X = rFFT_N(x_i block)
//                 C = sum_j conj(Hc_ij) G_jb               folded straight into
//                                                          the inverse pre-processing
//                 W_j += conj(X) G_jb
//                 c = irFFT_N(C)[0, hop): dx_i = alpha_i c, dalpha_i += <c, x_i>
//   then dh partial_ij = irFFT_N(W_j)[0, L_ij).
// A block costs J + 2I transforms.  Each thread owns the same bin pairs in
// every split and product, so its slots of G are private; x and g blocks, the
// source's RIR spectra and the block's G are staged with cp.async one step
// ahead of their use.  Microphones go in groups of kJG (the source spectra
// are recomputed per group; dx of later groups is added to the first
// group's).
template <int M>
struct BwdCfg {
    static constexpr int E = e_for(M);
    static constexpr int T = M / E;
    static constexpr bool kStage = M <= 4096;     // spectra and G staged in shared memory
    static constexpr bool kTwSmem = M <= 4096;
    static constexpr int kMinBlocks = M <= 2048 ? 2 : 1;
    static constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t o_sm = 0;
    static constexpr size_t o_xs = a16(o_sm + sizeof(float2) * padded_len(M));
    static constexpr size_t o_hs = a16(o_xs + sizeof(float) * 2 * M);
    static constexpr size_t o_gs = a16(o_hs + (kStage ? sizeof(float2) * kJG * M : 0));
    static constexpr size_t o_tw = a16(o_gs + (kStage ? sizeof(float2) * kJG * M : 0));
    static constexpr size_t bytes = a16(o_tw + (kTwSmem ? sizeof(float2) * FftPlan<M, E>::TW_LEN : 0));
};

template <int M>
__global__ void __launch_bounds__(BwdCfg<M>::T, BwdCfg<M>::kMinBlocks)
k_backward(DevBatch B, Queues Q, int bucket, const float* __restrict__ gy, const float* __restrict__ x,
           const float* __restrict__ gains, const float2* __restrict__ Hc, float* __restrict__ dx,
           float* __restrict__ dhp, float* __restrict__ dap, float2* __restrict__ Gc, int gc_blocks,
           const float2* __restrict__ twg) {
    using L = BwdCfg<M>;
    constexpr int E = L::E;
    constexpr int T = L::T;
    using Pl = FftPlan<M, E>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw + L::o_sm);
    float* xs = reinterpret_cast<float*>(smem_raw + L::o_xs);
    float2* hs = reinterpret_cast<float2*>(smem_raw + L::o_hs);
    float2* gs = reinterpret_cast<float2*>(smem_raw + L::o_gs);
    __shared__ double sd[32];
    __shared__ double dsum[kMaxSources];
    __shared__ int slot;
    const int t = threadIdx.x;
    const float2* tw = twg;
    if constexpr (L::kTwSmem) {
        float2* tws = reinterpret_cast<float2*>(smem_raw + L::o_tw);
        for (int k = t; k < Pl::TW_LEN; k += T) tws[k] = twg[k];
        __syncthreads();
        tw = tws;
    }
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    // this CTA's G slice: block bb, mic jj, slot e of thread t at ((bb kJG + jj) E + e) T + t
    float2* Gcta = Gc + (int64_t)blockIdx.x * gc_blocks * kJG * M;
    for (;;) {
        const int g = pop_job_b(Q, kListBwd, bucket, &slot);
        if (g < 0) break;
        const int u = B.bseg_utt[g];
        const int64_t sgi = g - B.bseg0[u];
        const int64_t nx = B.n_x[u];
        const int hop = B.hop[u];
        const int lmax = B.Lmax[u];
        int64_t b0, b1;
        segment_blocks(sgi, B.bseg_len, hop, B.nblk[u], &b0, &b1);
        if (b0 >= b1) continue;
        const int J = B.J, I = B.n_src[u];
        const int sb = B.src0[u], rb = B.rir0[u];
        if (t < kMaxSources) dsum[t] = 0.0;
        auto stage_x = [&](int i, int64_t b) {
            const int64_t p = b * hop;
            stage_real_async<M, E>(xs, x + B.xoff[sb + i] + p, min((int64_t)hop, nx - p), t);
        };
        auto stage_g = [&](int64_t b, int j) {
            const int64_t p = b * hop;
            stage_real_async<M, E>(xs, gy + B.yoff[u] + (int64_t)j * nx + p,
                                   min((int64_t)(hop + lmax - 1), nx - p), t);
        };
        auto gslot = [&](int64_t b, int jj) { return Gcta + ((b - b0) * kJG + jj) * (int64_t)M; };
        for (int j0 = 0; j0 < J; j0 += kJG) {
            const int jn = min(kJG, J - j0);
            // ---- phase 1: mic spectra of every block of the segment
            __syncthreads();                     // stages are free
            stage_g(b0, j0);
            cp_async_commit();
            for (int64_t b = b0; b < b1; ++b) {
                for (int jj = 0; jj < jn; ++jj) {
                    cp_async_wait<0>();
                    __syncthreads();
                    float2 v[E];
                    load_staged_strided<M, E>(v, xs, t);
                    __syncthreads();
                    if (jj + 1 < jn) stage_g(b, j0 + jj + 1);
                    else if (b + 1 < b1) stage_g(b + 1, j0);
                    else stage_x(0, b0);             // phase 2 starts with source 0, block b0
                    cp_async_commit();
                    rfft_regs_to_smem<M, E>(v, sm, tw, t);
                    float2* G = gslot(b, jj) + t;
#pragma unroll
                    for (int q = 0; q < E / 2; ++q)
                        split_pair<M>(sm, wsplit, t + q * T, G[(2 * q) * T], G[(2 * q + 1) * T]);
                }
            }
            __syncthreads();                     // G written by every thread is visible
            // ---- phase 2: per source
            for (int i = 0; i < I; ++i) {
                const float a = __ldg(gains + sb + i);
                const float* xi = x + B.xoff[sb + i];
                float* dxi = dx ? dx + B.xoff[sb + i] : nullptr;
                float da = 0.f, dac = 0.f;       // Kahan sum of c * x
                if constexpr (L::kStage) {
                    for (int jj = 0; jj < jn; ++jj) {
                        stage_spectrum_async<M, E>(hs + jj * M, Hc + (int64_t)(rb + i * J + j0 + jj) * B.MMAX, t);
                        stage_spectrum_async<M, E>(gs + jj * M, gslot(b0, jj), t);
                    }
                    cp_async_commit();
                }
                float2 W[kJG][E];
#pragma unroll
                for (int jj = 0; jj < kJG; ++jj)
#pragma unroll
                    for (int e = 0; e < E; ++e) W[jj][e] = make_float2(0.f, 0.f);
                for (int64_t b = b0; b < b1; ++b) {
                    const int64_t pos = b * hop;
                    const int64_t lim = nx - pos;
                    cp_async_wait<0>();
                    __syncthreads();
                    float2 v[E];
                    load_staged_strided<M, E>(v, xs, t);
                    __syncthreads();
                    if (b + 1 < b1) stage_x(i, b + 1);
                    else if (i + 1 < I) stage_x(i + 1, b0);
                    cp_async_commit();
                    rfft_regs_to_smem<M, E>(v, sm, tw, t);
                    float2 X[E];
                    split_forward<M, E>(X, sm, wsplit, t);
                    cp_async_wait<1>();          // spectra and G of this block are in
                    __syncthreads();             // (and every thread is done with sm)
#pragma unroll
                    for (int q = 0; q < E / 2; ++q) {
                        const int k = t + q * T;
                        const int kb = (k == 0) ? M / 2 : M - k;
                        float2 ca = make_float2(0.f, 0.f), cb = make_float2(0.f, 0.f);
#pragma unroll
                        for (int jj = 0; jj < kJG; ++jj) {
                            if (jj >= jn) break;
                            float2 ga, gb, ha, hb;
                            if constexpr (L::kStage) {
                                ga = gs[jj * M + (2 * q) * T + t];
                                gb = gs[jj * M + (2 * q + 1) * T + t];
                                ha = hs[jj * M + k];
                                hb = hs[jj * M + kb];
                            } else {
                                const float2* G = gslot(b, jj) + t;
                                ga = G[(2 * q) * T];
                                gb = G[(2 * q + 1) * T];
                                const float2* H = Hc + (int64_t)(rb + i * J + j0 + jj) * B.MMAX;
                                ha = __ldg(H + k);
                                hb = __ldg(H + kb);
                            }
                            if (k == 0) {            // slot 0 holds two real bins
                                ca.x += ha.x * ga.x;
                                ca.y += ha.y * ga.y;
                                W[jj][0].x += X[0].x * ga.x;
                                W[jj][0].y += X[0].y * ga.y;
                            } else {
                                ca = cadd(ca, cmulc(ha, ga));
                                W[jj][2 * q] = cadd(W[jj][2 * q], cmulc(X[2 * q], ga));
                            }
                            cb = cadd(cb, cmulc(hb, gb));
                            W[jj][2 * q + 1] = cadd(W[jj][2 * q + 1], cmulc(X[2 * q + 1], gb));
                        }
                        unsplit_pair<M>(sm, wsplit, k, ca, cb);
                    }
                    __syncthreads();             // gs fully read, sm fully written
                    if constexpr (L::kStage) {
                        if (b + 1 < b1) {
                            for (int jj = 0; jj < jn; ++jj) stage_spectrum_async<M, E>(gs + jj * M, gslot(b + 1, jj), t);
                        }
                        cp_async_commit();
                    }
                    irfft_from_smem<M, E>(v, sm, tw, t);
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int nn = n + e;
                            if (nn < hop && nn < lim) {
                                const float c = e ? v[q].y : v[q].x;
                                if (dxi) {
                                    const float d = a * c;
                                    dxi[pos + nn] = (j0 == 0) ? d : dxi[pos + nn] + d;
                                }
                                const float yv = fmaf(c, __ldg(xi + pos + nn), -dac);
                                const float tv = da + yv;
                                dac = (tv - da) - yv;
                                da = tv;
                            }
                        }
                    }
                }
                // dh partials of source i for mics j0 .. j0 + jn - 1
#pragma unroll
                for (int jj = 0; jj < kJG; ++jj) {
                    if (jj >= jn) break;
                    float2 v[E];
                    irfft_pairs<M, E>(v, W[jj], sm, tw, t);
                    const int r = rb + i * J + j0 + jj;
                    const int Lr = B.L[r];
                    float* out = dhp + B.dhp_off[g] + (B.roff[r] - B.roff[rb]);
#pragma unroll
                    for (int q = 0; q < E; ++q) {
                        const int n = 2 * (t + q * T);
                        if (n < Lr) out[n] = v[q].x;
                        if (n + 1 < Lr) out[n + 1] = v[q].y;
                    }
                }
                const double tot = block_sum_d((double)da - (double)dac, sd);
                if (t == 0) dsum[i] += tot;
            }
        }
        __syncthreads();
        if (t < I) dap[(int64_t)g * kMaxSources + t] = (float)dsum[t];
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// K8: deterministic reduction of the per-segment partials
// ---------------------------------------------------------------------------
// grad_rir[r][k] = alpha_i / N * sum_segments partial[k] for k < L_r, 0 for
// L_r <= k < Nh; grad_gains[s] = sum_segments dalpha partial.  Segments are
// added in order; empty segments (no block starts in them) are skipped.
__global__ void __launch_bounds__(256)
k_finalize(DevBatch B, const float* __restrict__ gains, const float* __restrict__ dhp,
           const float* __restrict__ dap, float* __restrict__ grad_rir, float* __restrict__ grad_gains) {
    for (int r = blockIdx.x; r < B.R; r += gridDim.x) {
        int lo = 0, hi = B.U - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (B.rir0[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const int u = lo;
        const int i = (r - B.rir0[u]) / B.J;
        const int Lr = B.L[r], nh = B.rir_len[r];
        float* out = grad_rir + B.roff[r];
        if (B.logN[u] == 0) {
            for (int k = threadIdx.x; k < nh; k += blockDim.x) out[k] = 0.f;
            continue;
        }
        const float scale = gains[B.src0[u] + i] / (float)(1 << B.logN[u]);
        const int64_t local = B.roff[r] - B.roff[B.rir0[u]];
        const int hop = B.hop[u];
        for (int k = threadIdx.x; k < nh; k += blockDim.x) {
            float acc = 0.f;
            if (k < Lr) {
                for (int g = B.bseg0[u]; g < B.bseg0[u + 1]; ++g) {
                    int64_t b0, b1;
                    segment_blocks(g - B.bseg0[u], B.bseg_len, hop, B.nblk[u], &b0, &b1);
                    if (b0 >= b1) continue;
                    acc += dhp[B.dhp_off[g] + local + k];
                }
            }
            out[k] = scale * acc;
        }
    }
    if (grad_gains) {
        for (int sidx = blockIdx.x * blockDim.x + threadIdx.x; sidx < B.S; sidx += gridDim.x * blockDim.x) {
            int lo = 0, hi = B.U - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (B.src0[mid] <= sidx) lo = mid; else hi = mid - 1;
            }
            const int u = lo, i = sidx - B.src0[u];
            float acc = 0.f;
            if (B.logN[u] != 0) {
                for (int g = B.bseg0[u]; g < B.bseg0[u + 1]; ++g) {
                    int64_t b0, b1;
                    segment_blocks(g - B.bseg0[u], B.bseg_len, B.hop[u], B.nblk[u], &b0, &b1);
                    if (b0 >= b1) continue;
                    acc += dap[(int64_t)g * kMaxSources + i];
                }
            }
            grad_gains[sidx] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int M>
constexpr int smem_backward() { return (int)BwdCfg<M>::bytes; }

template <int M>
static void backward_m(const DevBatch& B, const Queues& Q, int bucket, const float* g, const float* x,
                       const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                       float2* Gc, int gc_blocks, Twiddles tw, int grid, cudaStream_t st) {
    k_backward<M><<<grid, BwdCfg<M>::T, smem_backward<M>(), st>>>(B, Q, bucket, g, x, gains, Hc, dx, dhp,
                                                                  dap, Gc, gc_blocks, tw.get(BwdCfg<M>::E));
}

void launch_backward(int logN, const DevBatch& B, const Queues& Q, const float* g, const float* x,
                     const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                     float2* Gc, int gc_blocks, Twiddles tw, int grid, cudaStream_t st) {
    const int b = logN - kMinLog;
    switch (logN) {
        case 11: backward_m<1024>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, Gc, gc_blocks, tw, grid, st); break;
        case 12: backward_m<2048>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, Gc, gc_blocks, tw, grid, st); break;
        case 13: backward_m<4096>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, Gc, gc_blocks, tw, grid, st); break;
        case 14: backward_m<8192>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, Gc, gc_blocks, tw, grid, st); break;
        default: break;
    }
}

int bwd_threads(int logN) {
    switch (logN) {
        case 11: return BwdCfg<1024>::T;
        case 12: return BwdCfg<2048>::T;
        case 13: return BwdCfg<4096>::T;
        case 14: return BwdCfg<8192>::T;
    }
    return 1;
}

void launch_finalize(const DevBatch& B, const float* gains, const float* dhp, const float* dap,
                     float* grad_rir, float* grad_gains, cudaStream_t st) {
    int grid = B.R < 4096 ? B.R : 4096;
    if (grid < 1) grid = 1;
    k_finalize<<<grid, 256, 0, st>>>(B, gains, dhp, dap, grad_rir, grad_gains);
}

template <typename K>
static int occ_b(K kernel, int threads, int smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
    return n > 0 ? n : 1;
}

int occupancy_backward(int logN) {
    switch (logN) {
        case 11: return occ_b(k_backward<1024>, BwdCfg<1024>::T, smem_backward<1024>());
        case 12: return occ_b(k_backward<2048>, BwdCfg<2048>::T, smem_backward<2048>());
        case 13: return occ_b(k_backward<4096>, BwdCfg<4096>::T, smem_backward<4096>());
        case 14: return occ_b(k_backward<8192>, BwdCfg<8192>::T, smem_backward<8192>());
    }
    return 1;
}

}  // namespace rsim
