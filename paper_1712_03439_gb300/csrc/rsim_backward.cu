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
// Per block b of the segment:
//   G_j = rFFT_N(g_j[b hop, b hop + hop + L_max - 1))    once per mic, kept in
//                                                         shared memory (pair layout)
//   for each source i:
//     X_i = rFFT_N(x_i block)                             registers (pair layout)
//     C_i = sum_j conj(Hc_ij) G_j                          registers
//     W_ij += conj(X_i) G_j                                per-CTA scratch in L2
//     c_i = irFFT_N(C_i)[0, hop): dx_i = alpha_i c_i, dalpha_i += <c_i, x_i>
// so a block costs J + 2I transforms.  At the end of the segment
// dh partial_ij = irFFT_N(W_ij)[0, L_ij).  Each thread owns the same bin pairs
// in every split, product and pre-processing step, so its slots in G and W
// are private: no conflicts, no barriers around them.  Microphones go in
// groups of kJG (the source spectra are recomputed per group; dx of later
// groups is added to the first group's).
template <int M>
__global__ void __launch_bounds__(M / kE, (M <= 4096 ? 2 : 1))
k_backward(DevBatch B, Queues Q, int bucket, const float* __restrict__ gy, const float* __restrict__ x,
           const float* __restrict__ gains, const float2* __restrict__ Hc, float* __restrict__ dx,
           float* __restrict__ dhp, float* __restrict__ dap, float2* __restrict__ Wg,
           const float2* __restrict__ tw) {
    using Pl = FftPlan<M>;
    constexpr int T = M / kE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    float2* Gs = reinterpret_cast<float2*>(smem_raw + sizeof(float2) * padded_len(M)) + threadIdx.x;
    __shared__ double sd[32];
    __shared__ double dsum[kMaxSources];
    __shared__ int slot;
    const int t = threadIdx.x;
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    const int J = B.J;
    // this CTA's accumulators: W_ij slot e of thread t at ((i J + j) M + e T + t)
    float2* Wc = Wg + (int64_t)blockIdx.x * B.IMAX * J * M + t;
    for (;;) {
        const int g = pop_job_b(Q, kListBwd, bucket, &slot);
        if (g < 0) break;
        const int u = B.bseg_utt[g];
        const int64_t s = g - B.bseg0[u];
        const int64_t nx = B.n_x[u];
        const int hop = B.hop[u];
        const int lmax = B.Lmax[u];
        int64_t b0, b1;
        segment_blocks(s, B.bseg_len, hop, B.nblk[u], &b0, &b1);
        if (b0 >= b1) continue;
        const int I = B.n_src[u];
        const int sb = B.src0[u], rb = B.rir0[u];
        if (t < kMaxSources) dsum[t] = 0.0;
        for (int ij = 0; ij < I * J; ++ij)
#pragma unroll
            for (int e = 0; e < kE; ++e) Wc[(int64_t)ij * M + e * T] = make_float2(0.f, 0.f);
        for (int j0 = 0; j0 < J; j0 += kJG) {
            const int jn = min(kJG, J - j0);
            for (int64_t b = b0; b < b1; ++b) {
                const int64_t pos = b * hop;
                const int64_t len = min((int64_t)hop, nx - pos);
                const int64_t wlen = min((int64_t)(hop + lmax - 1), nx - pos);
                const int64_t lim = nx - pos;
                // mic spectra of this block
#pragma unroll
                for (int jj = 0; jj < kJG; ++jj) {
                    if (jj >= jn) break;
                    rfft_to_smem<M>(gy + B.yoff[u] + (int64_t)(j0 + jj) * nx + pos, wlen, sm, tw, t);
#pragma unroll
                    for (int q = 0; q < kE / 2; ++q)
                        split_pair<M>(sm, wsplit, t + q * T, Gs[(jj * kE + 2 * q) * T],
                                      Gs[(jj * kE + 2 * q + 1) * T]);
                }
                for (int i = 0; i < I; ++i) {
                    const float* xi = x + B.xoff[sb + i];
                    float2 X[kE];
                    rfft_to_smem<M>(xi + pos, len, sm, tw, t);
                    split_forward<M>(X, sm, wsplit, t);
                    float2 C[kE];
#pragma unroll
                    for (int e = 0; e < kE; ++e) C[e] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int jj = 0; jj < kJG; ++jj) {
                        if (jj >= jn) break;
                        const float2* H = Hc + (int64_t)(rb + i * J + j0 + jj) * B.MMAX;
                        float2* W = Wc + (int64_t)(i * J + j0 + jj) * M;
#pragma unroll
                        for (int q = 0; q < kE / 2; ++q) {
                            const int k = t + q * T;
                            const int kb = (k == 0) ? M / 2 : M - k;
                            const float2 ga = Gs[(jj * kE + 2 * q) * T], gb = Gs[(jj * kE + 2 * q + 1) * T];
                            const float2 ha = __ldg(H + k), hb = __ldg(H + kb);
                            float2 w0 = W[(2 * q) * T], w1 = W[(2 * q + 1) * T];
                            if (k == 0) {            // slot 0 holds two real bins
                                C[0].x += ha.x * ga.x;
                                C[0].y += ha.y * ga.y;
                                w0.x += X[0].x * ga.x;
                                w0.y += X[0].y * ga.y;
                            } else {
                                C[2 * q] = cadd(C[2 * q], cmulc(ha, ga));
                                w0 = cadd(w0, cmulc(X[2 * q], ga));
                            }
                            C[2 * q + 1] = cadd(C[2 * q + 1], cmulc(hb, gb));
                            w1 = cadd(w1, cmulc(X[2 * q + 1], gb));
                            W[(2 * q) * T] = w0;
                            W[(2 * q + 1) * T] = w1;
                        }
                    }
                    float2 v[kE];
                    irfft_pairs<M>(v, C, sm, tw, t);
                    const float a = __ldg(gains + sb + i);
                    float* dxi = dx ? dx + B.xoff[sb + i] : nullptr;
                    float da = 0.f, dac = 0.f;   // Kahan sum of c * x over this block
#pragma unroll
                    for (int q = 0; q < kE; ++q) {
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
                    const double tot = block_sum_d((double)da - (double)dac, sd);
                    if (t == 0) dsum[i] += tot;
                }
            }
        }
        // dh partials of this segment
        for (int ij = 0; ij < I * J; ++ij) {
            const float2* W = Wc + (int64_t)ij * M;
            __syncthreads();                 // sm is free
#pragma unroll 2
            for (int q = 0; q < kE / 2; ++q)
                unsplit_pair<M>(sm, wsplit, t + q * T, W[(2 * q) * T], W[(2 * q + 1) * T]);
            __syncthreads();
            float2 v[kE];
            irfft_from_smem<M>(v, sm, tw, t);
            const int r = rb + ij;
            const int Lr = B.L[r];
            float* out = dhp + B.dhp_off[g] + (B.roff[r] - B.roff[rb]);
#pragma unroll
            for (int q = 0; q < kE; ++q) {
                const int n = 2 * (t + q * T);
                if (n < Lr) out[n] = v[q].x;
                if (n + 1 < Lr) out[n + 1] = v[q].y;
            }
        }
        __syncthreads();
        if (t < I) dap[(int64_t)g * kMaxSources + t] = (float)dsum[t];
    }
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
constexpr int smem_backward() { return (int)sizeof(float2) * (padded_len(M) + kJG * M); }

template <int M>
static void backward_m(const DevBatch& B, const Queues& Q, int bucket, const float* g, const float* x,
                       const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                       float2* W, const float2* tw, int grid, cudaStream_t st) {
    k_backward<M><<<grid, M / kE, smem_backward<M>(), st>>>(B, Q, bucket, g, x, gains, Hc, dx, dhp,
                                                            dap, W, tw);
}

void launch_backward(int logN, const DevBatch& B, const Queues& Q, const float* g, const float* x,
                     const float* gains, const float2* Hc, float* dx, float* dhp, float* dap,
                     float2* W, const float2* tw, int grid, cudaStream_t st) {
    const int b = logN - kMinLog;
    switch (logN) {
        case 11: backward_m<1024>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, W, tw, grid, st); break;
        case 12: backward_m<2048>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, W, tw, grid, st); break;
        case 13: backward_m<4096>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, W, tw, grid, st); break;
        case 14: backward_m<8192>(B, Q, b, g, x, gains, Hc, dx, dhp, dap, W, tw, grid, st); break;
        default: break;
    }
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
        case 11: return occ_b(k_backward<1024>, 64, smem_backward<1024>());
        case 12: return occ_b(k_backward<2048>, 128, smem_backward<2048>());
        case 13: return occ_b(k_backward<4096>, 256, smem_backward<4096>());
        case 14: return occ_b(k_backward<8192>, 512, smem_backward<8192>());
    }
    return 1;
}

}  // namespace rsim
