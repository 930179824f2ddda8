// Block-level FFT building blocks for the overlap-add filter (sm_103a, FP32).
//
// A real N-point transform is computed as a complex M = N/2-point transform of
// z[n] = x[2n] + i x[2n+1] followed by the even/odd split (the "half spectrum"
// of Sec. 2.2: only bins 0..N/2 are kept, Hermitian symmetry gives the rest).
//
// The complex transform is a Stockham auto-sort FFT run by a CTA of T = M/E
// threads, each holding E complex values in registers.  Passes of radix E
// (the last one possibly smaller) run in registers and exchange through one
// padded shared-memory buffer.  Between passes thread t holds indices
// t + s*T, s < E ("strided layout"), which is both the load pattern of every
// pass and the output pattern of the last pass, so the last pass never touches
// shared memory.
//
// Twiddles come from tables built on the host in FP64 and rounded once to
// FP32 (no fast-math intrinsics): each pass stores the powers w^(2^j) and the
// other powers are products of a few of them.  The tables may sit in global
// or (copied once per CTA) shared memory.  The inverse transform is computed
// as conj(FFT(conj(.))) so one code path serves both directions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsim {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// a * (-i)
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }
// a * (+i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// small DFTs in registers, natural-order output, forward sign (e^{-2 pi i nk/R})
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_mi(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// cos and sin of 2*pi*e/16 for e = 1, 2, 3
#define RSIM_C1 0.92387953251128675613f
#define RSIM_S1 0.38268343236508977173f
#define RSIM_R2 0.70710678118654752440f

// multiply by w16^e = e^{-2 pi i e / 16} for the exponents a 16-point
// transform needs (e in {0, 1, 2, 3, 4, 6, 9})
template <int e>
__device__ __forceinline__ float2 w16(float2 a) {
    if constexpr (e == 0) return a;
    else if constexpr (e == 1) return cmul(a, make_float2(RSIM_C1, -RSIM_S1));
    else if constexpr (e == 2) return make_float2(RSIM_R2 * (a.x + a.y), RSIM_R2 * (a.y - a.x));
    else if constexpr (e == 3) return cmul(a, make_float2(RSIM_S1, -RSIM_C1));
    else if constexpr (e == 4) return mul_mi(a);
    else if constexpr (e == 6) return make_float2(RSIM_R2 * (a.y - a.x), -RSIM_R2 * (a.x + a.y));
    else if constexpr (e == 9) return cmul(a, make_float2(-RSIM_C1, RSIM_S1));
    else return a;  // unused
}

__device__ __forceinline__ void dft8(float2 (&a)[8]) {
    // n = 2 n1 + n2, k = k1 + 4 k2
    dft4(a[0], a[2], a[4], a[6]);
    dft4(a[1], a[3], a[5], a[7]);
    // twiddle w8^{n2 k1} = w16^{2 k1} on the odd half
    a[3] = w16<2>(a[3]);
    a[5] = w16<4>(a[5]);
    a[7] = w16<6>(a[7]);
    float2 b[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 e = a[2 * k1], o = a[2 * k1 + 1];
        b[k1] = cadd(e, o);
        b[k1 + 4] = csub(e, o);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = b[k];
}

__device__ __forceinline__ void dft16(float2 (&a)[16]) {
    // n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    // now a[n2 + 4 k1] = B[n2][k1]; twiddle by w16^{n2 k1}
    a[5] = w16<1>(a[5]);
    a[9] = w16<2>(a[9]);
    a[13] = w16<3>(a[13]);
    a[6] = w16<2>(a[6]);
    a[10] = w16<4>(a[10]);
    a[14] = w16<6>(a[14]);
    a[7] = w16<3>(a[7]);
    a[11] = w16<6>(a[11]);
    a[15] = w16<9>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // a[4 k1 + k2] = A[k1 + 4 k2]: transpose the 4x4 index
    float2 b[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) b[k1 + 4 * k2] = a[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = b[k];
}

template <int R>
__device__ __forceinline__ void dft(float2 (&u)[R]) {
    if constexpr (R == 2) dft2(u[0], u[1]);
    else if constexpr (R == 4) dft4(u[0], u[1], u[2], u[3]);
    else if constexpr (R == 8) dft8(u);
    else dft16(u);
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// values per thread for a complex size M
__host__ __device__ constexpr int e_for(int M) { return 8; }

// padded shared-memory index: one spare float2 every 16.  With T a multiple
// of 16 the strided loads and stores are conflict-free, and so are the
// scatter stores of the radix-16 passes and of the radix-8 passes except
// the one with LP = 8 (2-way on part of its lanes).
__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int M) { return M + (M >> 4); }

template <int M, int E = e_for(M)>
struct FftPlan {
    static constexpr int T = M / E;
    static constexpr int LOGE = ilog2(E);
    static constexpr int LOGM = ilog2(M);
    static constexpr int NPASS = (LOGM + LOGE - 1) / LOGE;
    static constexpr int R_LAST = 1 << (LOGM - (NPASS - 1) * LOGE);
    static constexpr int radix(int p) { return p < NPASS - 1 ? E : R_LAST; }
    static constexpr int lp(int p) { return 1 << (p * LOGE); }   // product of the earlier radices
    // Twiddle table: pass p >= 1 stores log2(radix(p)) rows of lp(p) entries,
    // row j holding w^(2^j) = exp(-2 pi i 2^j k / (lp(p) radix(p))), k < lp(p);
    // then the split table exp(-2 pi i k / (2M)), k <= M/2.
    static constexpr int tw_off(int p) {
        return p <= 1 ? 0 : tw_off(p - 1) + ilog2(radix(p - 1)) * lp(p - 1);
    }
    static constexpr int OFF_SPLIT = tw_off(NPASS);
    static constexpr int TW_LEN = OFF_SPLIT + M / 2 + 1;
    static_assert(T % 16 == 0, "T must be a multiple of 16");
};

// u[m] *= w^m, m = 1 .. R-1, from the power rows of a pass table
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 (&u)[R], const float2* __restrict__ tab, int LP, int k) {
    const float2 w1 = tab[k];
    if constexpr (R == 2) {
        u[1] = cmul(u[1], w1);
    } else {
        const float2 w2 = tab[LP + k];
        const float2 w3 = cmul(w1, w2);
        u[1] = cmul(u[1], w1);
        u[2] = cmul(u[2], w2);
        u[3] = cmul(u[3], w3);
        if constexpr (R >= 8) {
            const float2 w4 = tab[2 * LP + k];
            u[4] = cmul(u[4], w4);
            u[5] = cmul(u[5], cmul(w4, w1));
            u[6] = cmul(u[6], cmul(w4, w2));
            const float2 w7 = cmul(w4, w3);
            u[7] = cmul(u[7], w7);
            if constexpr (R == 16) {
                const float2 w8 = tab[3 * LP + k];
                u[8] = cmul(u[8], w8);
                u[9] = cmul(u[9], cmul(w8, w1));
                u[10] = cmul(u[10], cmul(w8, w2));
                u[11] = cmul(u[11], cmul(w8, w3));
                u[12] = cmul(u[12], cmul(w8, w4));
                u[13] = cmul(u[13], cmul(w8, cmul(w4, w1)));
                u[14] = cmul(u[14], cmul(w8, cmul(w4, w2)));
                u[15] = cmul(u[15], cmul(w8, w7));
            }
        }
    }
}

// padded offset of element base + m * LP relative to pad(base), for the
// scatter of a Stockham pass (base = (i - k) R + k with k < LP)
template <int LP>
__device__ __forceinline__ constexpr int scatter_off(int m) {
    if constexpr (LP >= 16) return m * (LP + LP / 16);
    else if constexpr (LP == 8) return 8 * m + (m >> 1);   // base % 16 = k < 8
    else return m * LP;                                    // LP = 1: base % 16 + m < 16
}

// One Stockham pass of radix R with LP = product of the earlier radices.
// Input: v in strided layout.  If LAST, the output stays in v (strided);
// otherwise it is scattered to shared memory.
template <int M, int E, int R, int LP, bool LAST>
__device__ __forceinline__ void fft_pass(float2 (&v)[E], float2* __restrict__ sm,
                                         const float2* __restrict__ tw, int t) {
    constexpr int T = M / E;
    constexpr int NB = E / R;  // butterflies per thread
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        float2 u[R];
#pragma unroll
        for (int m = 0; m < R; ++m) u[m] = v[q + m * NB];
        const int i = t + q * T;
        const int k = i & (LP - 1);
        if constexpr (LP > 1) apply_twiddles<R>(u, tw, LP, k);
        dft<R>(u);
        if constexpr (LAST) {
#pragma unroll
            for (int m = 0; m < R; ++m) v[q + m * NB] = u[m];
        } else {
            float2* dst = sm + pad((i - k) * R + k);
#pragma unroll
            for (int m = 0; m < R; ++m) dst[scatter_off<LP>(m)] = u[m];
        }
    }
}

template <int M, int E>
__device__ __forceinline__ void load_strided(float2 (&v)[E], const float2* __restrict__ sm, int t) {
    constexpr int T = M / E;
    const float2* src = sm + t + (t >> 4);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = src[s * (T + T / 16)];
}

template <int M, int E>
__device__ __forceinline__ void store_strided(const float2 (&v)[E], float2* __restrict__ sm, int t) {
    constexpr int T = M / E;
    float2* dst = sm + t + (t >> 4);
#pragma unroll
    for (int s = 0; s < E; ++s) dst[s * (T + T / 16)] = v[s];
}

// passes P .. NPASS-1; entered with v in strided layout and sm free
template <int M, int E, int P>
__device__ __forceinline__ void fft_from(float2 (&v)[E], float2* __restrict__ sm,
                                         const float2* __restrict__ tw, int t) {
    using Pl = FftPlan<M, E>;
    constexpr int R = Pl::radix(P), LP = Pl::lp(P);
    if constexpr (P == Pl::NPASS - 1) {
        fft_pass<M, E, R, LP, true>(v, sm, tw + Pl::tw_off(P), t);
    } else {
        fft_pass<M, E, R, LP, false>(v, sm, tw + Pl::tw_off(P), t);
        __syncthreads();
        load_strided<M, E>(v, sm, t);
        if constexpr (P + 2 < Pl::NPASS) __syncthreads();   // the next pass scatters in place
        fft_from<M, E, P + 1>(v, sm, tw, t);
    }
}

// Complex forward FFT of size M.  v: strided input in registers; on return v
// holds the spectrum in strided layout (natural bin index t + s*T).
// Starts with a __syncthreads so the caller may still be reading sm.
template <int M, int E>
__device__ __forceinline__ void fft_core(float2 (&v)[E], float2* __restrict__ sm,
                                         const float2* __restrict__ tw, int t) {
    __syncthreads();
    fft_from<M, E, 0>(v, sm, tw, t);
}

// ---------------------------------------------------------------------------
// real-signal helpers
// ---------------------------------------------------------------------------

// Loads z[n] = x[2n] + i x[2n+1] for the strided indices of thread t from a
// real segment src[0, len) in global memory (zero outside; src may be unaligned).
template <int M, int E>
__device__ __forceinline__ void load_real_strided(float2 (&v)[E], const float* __restrict__ src,
                                                  int64_t len, int t) {
    constexpr int T = M / E;
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const int64_t n = 2 * (int64_t)(t + s * T);
        float a = (n < len) ? __ldg(src + n) : 0.f;
        float b = (n + 1 < len) ? __ldg(src + n + 1) : 0.f;
        v[s] = make_float2(a, b);
    }
}

// Pair layout of a half spectrum: thread t owns, for s < E/2, bins
// k_s = t + s*T (k_s < M/2) and their mirrors M - k_s, in P[2s] and P[2s+1].
// Thread 0, s = 0 owns slot 0 -- (X[0], X[M]) packed as one float2 (both are
// real) -- in P[0], and the self-mirrored bin M/2 in P[1].

// Split of one pair: from Z = FFT_M(z) in shared memory (natural order,
// padded) to the true half spectrum of the real 2M-point signal:
// xa = X[k], xb = X[M-k]; for k = 0, xa = (X[0], X[M]) and xb = X[M/2].
// wsplit[k] = exp(-2 pi i k / (2M)).
// The mirror slot the split of bin k reads besides k itself: Z[M/2] for k = 0.
template <int M>
__host__ __device__ constexpr int split_mirror(int k) { return k == 0 ? M / 2 : M - k; }

// The split arithmetic on zk = Z[k] and zq = Z[split_mirror(k)].
template <int M>
__device__ __forceinline__ void split_values(float2 zk, float2 zq, const float2* __restrict__ wsplit,
                                             int k, float2& xa, float2& xb) {
    if (k == 0) {
        xa = make_float2(zk.x + zk.y, zk.x - zk.y);
        xb = conjf2(zq);
    } else {
        const float2 zm = conjf2(zq);
        const float2 E = cscale(cadd(zk, zm), 0.5f);
        const float2 O = cscale(mul_mi(csub(zk, zm)), 0.5f);   // (zk - zm) / (2i)
        const float2 wO = cmul(wsplit[k], O);
        xa = cadd(E, wO);
        xb = conjf2(csub(E, wO));
    }
}

template <int M>
__device__ __forceinline__ void split_pair(const float2* __restrict__ sm, const float2* __restrict__ wsplit,
                                           int k, float2& xa, float2& xb) {
    if (k == 0) split_values<M>(sm[pad(0)], sm[pad(M / 2)], wsplit, 0, xa, xb);
    else split_values<M>(sm[pad(k)], sm[pad(M - k)], wsplit, k, xa, xb);
}

// Split into pair layout registers P[2s] = X[k_s], P[2s+1] = X[M-k_s].
template <int M, int E>
__device__ __forceinline__ void split_forward(float2 (&P)[E], const float2* __restrict__ sm,
                                              const float2* __restrict__ wsplit, int t) {
    constexpr int T = M / E;
#pragma unroll
    for (int s = 0; s < E / 2; ++s) split_pair<M>(sm, wsplit, t + s * T, P[2 * s], P[2 * s + 1]);
}

// split_forward reading the buffer with volatile loads, for a spectrum kept in
// registers while later transforms of a rolled loop rewrite the same buffer
// (one exchange buffer: every transform's spectrum lands at the same address).
// With plain loads the compiled code was seen to produce, where the kept values
// are used, the split of what the buffer holds at that point -- as if the reads
// of one address in different iterations were one value across the barriers
// between them.  Volatile loads are each performed where they stand.
template <int M, int E>
__device__ __forceinline__ void split_forward_now(float2 (&P)[E], const float2* sm,
                                                  const float2* __restrict__ wsplit, int t) {
    constexpr int T = M / E;
    const volatile float2* vs = sm;
#pragma unroll
    for (int s = 0; s < E / 2; ++s) {
        const int k = t + s * T;
        const int a = pad(k), b = pad(split_mirror<M>(k));
        split_values<M>(make_float2(vs[a].x, vs[a].y), make_float2(vs[b].x, vs[b].y), wsplit, k,
                        P[2 * s], P[2 * s + 1]);
    }
}

// Inverse pre-processing of one pair: from ya = Y[k], yb = Y[M-k] (for k = 0:
// (Y[0], Y[M]) and Y[M/2]) of a half spectrum to conj(Z') in shared memory,
// where Z' = 2 FFT_M(z) of the signal y = IDFT_{2M}(Y) * 2M.  Running
// fft_core on it and conjugating gives z[n] = y[2n] + i y[2n+1] scaled by
// 2M (unnormalised inverse).
template <int M>
__device__ __forceinline__ void unsplit_pair(float2* __restrict__ sm, const float2* __restrict__ wsplit,
                                             int k, float2 ya, float2 yb) {
    if (k == 0) {
        sm[pad(0)] = conjf2(make_float2(ya.x + ya.y, ya.x - ya.y));
        sm[pad(M / 2)] = cscale(yb, 2.f);                  // conj(2 conj(Y[M/2]))
    } else {
        const float2 ym = conjf2(yb);
        const float2 E = cadd(ya, ym);
        const float2 D = csub(ya, ym);
        const float2 O = cmulc(wsplit[k], D);               // D * conj(w^k)
        const float2 zk = cadd(E, mul_pi(O));               // E + i O
        const float2 zm = cadd(conjf2(E), mul_pi(conjf2(O)));
        sm[pad(k)] = conjf2(zk);
        sm[pad(M - k)] = conjf2(zm);
    }
}

template <int M, int E>
__device__ __forceinline__ void split_inverse_store(const float2 (&P)[E], float2* __restrict__ sm,
                                                    const float2* __restrict__ wsplit, int t) {
    constexpr int T = M / E;
#pragma unroll
    for (int s = 0; s < E / 2; ++s) unsplit_pair<M>(sm, wsplit, t + s * T, P[2 * s], P[2 * s + 1]);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async, completion by groups)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 4 bytes, zero-filled when !valid (no global read then)
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0));
}
// 16 bytes; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Queues the copy of the real block src[0, len) into stage[0, 2M), zeros
// beyond len.  Thread t copies elements t + k*T (coalesced): rows wholly
// inside the block copy without a per-element predicate, the one ragged row
// is predicated, and rows past the block are zeroed with plain stores.
template <int M, int E>
__device__ __forceinline__ void stage_real_async(float* __restrict__ stage, const float* __restrict__ src,
                                                 int64_t len, int t) {
    constexpr int T = M / E;
    const int ilen = (int)(len < 2 * M ? (len > 0 ? len : 0) : 2 * M);
    const int kfull = ilen / T;                  // rows wholly inside the block
    float* d = stage + t;
    const float* s = src + t;
#pragma unroll 4
    for (int k = 0; k < kfull; ++k) cp_async4(d + k * T, s + k * T, true);
    if (kfull < 2 * E) {
        const bool ok = kfull * T + t < ilen;
        cp_async4(d + kfull * T, ok ? s + kfull * T : src, ok);
#pragma unroll 4
        for (int k = kfull + 1; k < 2 * E; ++k) d[k * T] = 0.f;
    }
}

// Queues the copy of M float2 from 16-byte aligned global memory into
// 16-byte aligned shared memory.
template <int M, int E>
__device__ __forceinline__ void stage_spectrum_async(float2* __restrict__ dst, const float2* __restrict__ src,
                                                     int t) {
    constexpr int T = M / E;
#pragma unroll
    for (int k = 0; k < M / 2 / T; ++k) {
        const int c = t + k * T;
        cp_async16(dst + 2 * c, src + 2 * c);
    }
}

// z[n] = (stage[2n], stage[2n+1]) for the strided indices of thread t
template <int M, int E>
__device__ __forceinline__ void load_staged_strided(float2 (&v)[E], const float* __restrict__ stage, int t) {
    constexpr int T = M / E;
    const float2* s2 = reinterpret_cast<const float2*>(stage);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = s2[t + s * T];
}

// ---------------------------------------------------------------------------
// bulk staging (the copy engine moves a block's whole 16-byte chunks)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* mb, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::); }
// orders this thread's earlier (generic) shared-memory accesses before its later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::); }
__device__ __forceinline__ void mbar_arrive(uint64_t* mb) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mb)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mb) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mb))
                 : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}
// Waits for the phase with the given parity to complete; gives up after about
// limit_ns of wall time and returns false then.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mb, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mb)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mb, uint32_t parity,
                                                  uint64_t limit_ns = 500000000ull) {
    if (mbar_try_wait(mb, parity)) return true;      // the usual case: the copy is in
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(mb, parity)) return true;
        if ((it & 63) == 0 && global_ns() - t0 > limit_ns) return false;
    }
}

// Queues the real block src[0, len) (zeros after it, len clipped to [0, 2M])
// into stage at float offset off = (src's float position within its 16-byte
// chunk), so that the whole chunks can move by one bulk copy (issued by
// thread 0, completing on mb); the at most three head and three tail floats
// and the zero fill are plain stores.  Every thread must call it, after a
// barrier that retired the stage's previous readers.  The stage holds
// 2M + 8 floats.  Returns off; read with load_staged_at after mb completes
// and a barrier has passed.
// (withhold: test hook -- the barrier is told to expect the bytes but no copy
// is issued, so the readers' bounded wait runs out)
template <int M, int E>
__device__ __forceinline__ int stage_real_bulk(float* __restrict__ stage, const float* __restrict__ src,
                                               int64_t len64, uint64_t* mb, int t, bool withhold = false) {
    constexpr int T = M / E;
    const int len = (int)(len64 < 2 * M ? (len64 > 0 ? len64 : 0) : 2 * M);
    const int off = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
    const int head = off ? min(len, 4 - off) : 0;
    const int body = ((len - head) >> 2) << 2;
    if (t == 0) {
        fence_proxy_async_smem();
        if (body > 0) {
            mbar_arrive_expect_tx(mb, (uint32_t)body * 4u);
            if (!withhold) bulk_copy_g2s(stage + off + head, src + head, (uint32_t)body * 4u, mb);
        } else {
            mbar_arrive(mb);
        }
    }
    if (t < head) stage[off + t] = __ldg(src + t);
    const int tail0 = head + body;
    if (t < len - tail0) stage[off + tail0 + t] = __ldg(src + tail0 + t);
    for (int n = len + t; n < 2 * M; n += T) stage[off + n] = 0.f;
    return off;
}

// z[n] = (stage[off + 2n], stage[off + 2n + 1]) for the strided indices of thread t
template <int M, int E>
__device__ __forceinline__ void load_staged_at(float2 (&v)[E], const float* __restrict__ stage, int off, int t) {
    constexpr int T = M / E;
    if ((off & 1) == 0) {
        const float2* s2 = reinterpret_cast<const float2*>(stage + off);
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = s2[t + s * T];
    } else {
        const float* s1 = stage + off;
#pragma unroll
        for (int s = 0; s < E; ++s) v[s] = make_float2(s1[2 * (t + s * T)], s1[2 * (t + s * T) + 1]);
    }
}

// ---------------------------------------------------------------------------
// composite real transforms
// ---------------------------------------------------------------------------

// FFT of strided registers v into sm (natural order); read pairs with
// split_pair afterwards.
template <int M, int E>
__device__ __forceinline__ void rfft_regs_to_smem(float2 (&v)[E], float2* __restrict__ sm,
                                                  const float2* __restrict__ tw, int t) {
    fft_core<M, E>(v, sm, tw, t);
    __syncthreads();                 // everyone done with the last pass loads
    store_strided<M, E>(v, sm, t);
    __syncthreads();
}

// Forward real FFT of src[0, len) (global) zero-padded to 2M, into pair layout P.
template <int M, int E>
__device__ __forceinline__ void rfft_pairs(float2 (&P)[E], const float* __restrict__ src, int64_t len,
                                           float2* __restrict__ sm, const float2* __restrict__ tw, int t) {
    float2 v[E];
    load_real_strided<M, E>(v, src, len, t);
    rfft_regs_to_smem<M, E>(v, sm, tw, t);
    split_forward<M, E>(P, sm, tw + FftPlan<M, E>::OFF_SPLIT, t);
}

// Inverse real FFT after the caller has written conj(Z') to sm with
// unsplit_pair and synchronised: v[s] = (y[2n], y[2n+1]) * 2M, n = t + s*T.
template <int M, int E>
__device__ __forceinline__ void irfft_from_smem(float2 (&v)[E], float2* __restrict__ sm,
                                                const float2* __restrict__ tw, int t) {
    load_strided<M, E>(v, sm, t);
    fft_core<M, E>(v, sm, tw, t);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = conjf2(v[s]);
}

// Unnormalised inverse real FFT of a half spectrum in pair layout.  On return
// v[s] holds (y[2n], y[2n+1]) * 2M for n = t + s*T.
template <int M, int E>
__device__ __forceinline__ void irfft_pairs(float2 (&v)[E], const float2 (&P)[E],
                                            float2* __restrict__ sm, const float2* __restrict__ tw, int t) {
    __syncthreads();                 // sm may still be read by a previous phase
    split_inverse_store<M, E>(P, sm, tw + FftPlan<M, E>::OFF_SPLIT, t);
    __syncthreads();
    load_strided<M, E>(v, sm, t);
    fft_core<M, E>(v, sm, tw, t);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = conjf2(v[s]);
}

// ---------------------------------------------------------------------------
// alternating exchange buffers
// ---------------------------------------------------------------------------
// Every shared-memory exchange of a transform is "write buffer, barrier, read
// buffer".  With two buffers used in strict alternation by every exchange of
// a kernel, the buffer an exchange writes was last read two exchanges earlier,
// before the previous exchange's barrier, so one barrier per exchange is
// enough.  With NB = 1 both slots are the same buffer and each exchange adds
// the barrier that protects its write.
template <int NB>
struct Exch {
    float2* b0;
    float2* b1;
    int c;
    __device__ __forceinline__ float2* begin() {
        if constexpr (NB == 1) __syncthreads();
        return c ? b1 : b0;
    }
    __device__ __forceinline__ void end() {
        if constexpr (NB == 2) c ^= 1;
    }
};

template <int M, int E, int P, int NB>
__device__ __forceinline__ void fft_from_x(float2 (&v)[E], Exch<NB>& ex, const float2* __restrict__ tw, int t) {
    using Pl = FftPlan<M, E>;
    constexpr int R = Pl::radix(P), LP = Pl::lp(P);
    if constexpr (P == Pl::NPASS - 1) {
        fft_pass<M, E, R, LP, true>(v, nullptr, tw + Pl::tw_off(P), t);
    } else {
        float2* b = ex.begin();
        fft_pass<M, E, R, LP, false>(v, b, tw + Pl::tw_off(P), t);
        __syncthreads();
        load_strided<M, E>(v, b, t);
        ex.end();
        fft_from_x<M, E, P + 1, NB>(v, ex, tw, t);
    }
}

// Forward FFT of strided registers v; returns the buffer holding the spectrum
// in natural order (read it with split_pair before the second exchange after
// this one).  With WAIT, the caller's outstanding cp.async groups complete
// before the last barrier, so data staged before the call is visible after it.
template <int M, int E, bool WAIT, int NB>
__device__ __forceinline__ const float2* rfft_x(float2 (&v)[E], Exch<NB>& ex, const float2* __restrict__ tw, int t) {
    fft_from_x<M, E, 0, NB>(v, ex, tw, t);
    float2* b = ex.begin();
    store_strided<M, E>(v, b, t);
    if constexpr (WAIT) cp_async_wait<0>();
    __syncthreads();
    ex.end();
    return b;
}

// Unnormalised inverse real FFT of a half spectrum in pair layout (see
// irfft_pairs); WAIT as for rfft_x.
template <int M, int E, bool WAIT, int NB>
__device__ __forceinline__ void irfft_x(float2 (&v)[E], const float2 (&P)[E], Exch<NB>& ex,
                                        const float2* __restrict__ tw, int t) {
    float2* b = ex.begin();
    split_inverse_store<M, E>(P, b, tw + FftPlan<M, E>::OFF_SPLIT, t);
    if constexpr (WAIT) cp_async_wait<0>();
    __syncthreads();
    load_strided<M, E>(v, b, t);
    ex.end();
    fft_from_x<M, E, 0, NB>(v, ex, tw, t);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = conjf2(v[s]);
}

// ---------------------------------------------------------------------------
// real split in registers (last pass of full radix)
// ---------------------------------------------------------------------------
// When every pass has radix E (M = E^k), the last forward pass can be given to
// the threads in an order that puts butterflies i and T - i (whose outputs
// hold the mirror bins k and M - k) in lanes l and l ^ 16 of one warp; the
// even/odd split then needs one register swap between those lanes instead of
// a trip through shared memory.  Butterflies 0 and T/2 mirror onto
// themselves.  The half spectrum comes out in "paired layout": thread t with
// butterfly i = paired_butterfly(t) holds P[2m] = X[k_m], P[2m+1] = X[M-k_m],
// k_m = i + T m, m < E/2 (k = 0: P[0] = (X[0], X[M]) packed, P[1] = X[M/2]).
// The inverse takes the same layout, swaps the mirror halves back and runs
// its first pass with butterfly i.
template <int M, int E>
struct PairedSplit {
    static constexpr bool ok = FftPlan<M, E>::R_LAST == E && (M / E) % 32 == 0;
};

template <int T>
__device__ __forceinline__ int paired_butterfly(int t) {
    const int w = t >> 5, l = t & 31;
    if (l < 16) return 16 * w + l;
    if (w == 0 && l == 16) return T / 2;
    return T - (16 * w + l - 16);
}

// forward passes P..; the last one runs butterfly i.  WAIT as for rfft_x,
// folded into the last exchange.
template <int M, int E, int P, bool WAIT, int NB>
__device__ __forceinline__ void fft_from_paired(float2 (&v)[E], Exch<NB>& ex, const float2* __restrict__ tw,
                                                int t, int i) {
    using Pl = FftPlan<M, E>;
    constexpr int R = Pl::radix(P), LP = Pl::lp(P);
    if constexpr (P == Pl::NPASS - 1) {
        fft_pass<M, E, R, LP, true>(v, nullptr, tw + Pl::tw_off(P), i);
    } else {
        float2* b = ex.begin();
        fft_pass<M, E, R, LP, false>(v, b, tw + Pl::tw_off(P), t);
        constexpr bool kLastExchange = P + 1 == Pl::NPASS - 1;
        if constexpr (WAIT && kLastExchange) cp_async_wait<0>();
        __syncthreads();
        load_strided<M, E>(v, b, kLastExchange ? i : t);
        ex.end();
        fft_from_paired<M, E, P + 1, WAIT, NB>(v, ex, tw, t, i);
    }
}

// The partner lane's mirror values pw[m] = partner's v[E-1-m], m < E/2.
template <int E>
__device__ __forceinline__ void paired_swap(float2 (&pw)[E / 2], const float2 (&v)[E]) {
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
        pw[m].x = __shfl_xor_sync(0xffffffffu, v[E - 1 - m].x, 16);
        pw[m].y = __shfl_xor_sync(0xffffffffu, v[E - 1 - m].y, 16);
    }
}

// Split of pair m in paired layout: xa = X[k_m], xb = X[M - k_m] (for k = 0:
// xa = (X[0], X[M]), xb = X[M/2]), from v[m] = Z[k_m] and the mirror value.
template <int M, int E>
__device__ __forceinline__ void paired_split_pair(const float2 (&v)[E], const float2 (&pw)[E / 2],
                                                  const float2* __restrict__ wsplit, int i, int m,
                                                  float2& xa, float2& xb) {
    constexpr int T = M / E;
    if (i == 0 && m == 0) {                 // bins 0, M and M/2 (all from this thread)
        const float2 z0 = v[0], zh = v[E / 2];
        xa = make_float2(z0.x + z0.y, z0.x - z0.y);
        xb = conjf2(zh);
        return;
    }
    const float2 zk = v[m];
    const float2 zm = conjf2((i == 0) ? v[E - m] : (i == T / 2 ? v[E - 1 - m] : pw[m]));
    const float2 Ev = cscale(cadd(zk, zm), 0.5f);
    const float2 Od = cscale(mul_mi(csub(zk, zm)), 0.5f);   // (zk - zm) / (2i)
    const float2 wO = cmul(wsplit[i + T * m], Od);
    xa = cadd(Ev, wO);
    xb = conjf2(csub(Ev, wO));
}

// The real split after the forward passes: paired layout P from v.
template <int M, int E>
__device__ __forceinline__ void paired_split(float2 (&P)[E], const float2 (&v)[E], const float2* __restrict__ tw,
                                             int i) {
    const float2* wsplit = tw + FftPlan<M, E>::OFF_SPLIT;
    float2 pw[E / 2];
    paired_swap<E>(pw, v);
#pragma unroll
    for (int m = 0; m < E / 2; ++m) paired_split_pair<M, E>(v, pw, wsplit, i, m, P[2 * m], P[2 * m + 1]);
}

// Forward real FFT of strided registers v into paired layout P.
template <int M, int E, bool WAIT, int NB>
__device__ __forceinline__ void rfft_paired(float2 (&P)[E], float2 (&v)[E], Exch<NB>& ex,
                                            const float2* __restrict__ tw, int t, int i) {
    static_assert(PairedSplit<M, E>::ok, "paired split needs M = E^k");
    fft_from_paired<M, E, 0, WAIT, NB>(v, ex, tw, t, i);
    paired_split<M, E>(P, v, tw, i);
}

// Passes P .. NPASS-1 of the complex FFT of strided registers, pass 0 running
// butterfly `first`, the last pass (and the exchange before it) butterfly
// `last` and every other pass t: (t, i) is the forward of the paired layout
// (as fft_from_paired), (i, t) the passes of the inverse (as irfft_paired) --
// one code path for both where a kernel alternates between them.
template <int M, int E, int P, int NB>
__device__ __forceinline__ void fft_passes_sel(float2 (&v)[E], Exch<NB>& ex, const float2* __restrict__ tw, int t,
                                               int first, int last) {
    using Pl = FftPlan<M, E>;
    constexpr int R = Pl::radix(P), LP = Pl::lp(P);
    static_assert(Pl::NPASS >= 2, "a first and a last pass");
    if constexpr (P == Pl::NPASS - 1) {
        fft_pass<M, E, R, LP, true>(v, nullptr, tw + Pl::tw_off(P), last);
    } else {
        float2* b = ex.begin();
        fft_pass<M, E, R, LP, false>(v, b, tw + Pl::tw_off(P), P == 0 ? first : t);
        constexpr bool kLastExchange = P + 1 == Pl::NPASS - 1;
        __syncthreads();
        load_strided<M, E>(v, b, kLastExchange ? last : t);
        ex.end();
        fft_passes_sel<M, E, P + 1, NB>(v, ex, tw, t, first, last);
    }
}

// Unnormalised inverse real FFT of a half spectrum in paired layout; on
// return v[s] holds (y[2n], y[2n+1]) * 2M for n = t + s*T (as irfft_pairs).
// The inverse's preparation of a half spectrum P in paired layout: on return v
// holds what the inverse's passes (pass 0 running butterfly i) transform.
template <int M, int E>
__device__ __forceinline__ void paired_unsplit(float2 (&v)[E], const float2 (&P)[E], const float2* __restrict__ tw,
                                               int i) {
    constexpr int T = M / E;
    using Pl = FftPlan<M, E>;
    const float2* wsplit = tw + Pl::OFF_SPLIT;
    float2 mir[E / 2];                      // conj(Z') at the mirror bins M - k_m
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
        if (i == 0 && m == 0) {
            const float2 ya = P[0], yb = P[1];
            v[0] = conjf2(make_float2(ya.x + ya.y, ya.x - ya.y));
            v[E / 2] = cscale(yb, 2.f);
            mir[0] = make_float2(0.f, 0.f);
            continue;
        }
        const int k = i + T * m;
        const float2 ya = P[2 * m], ym = conjf2(P[2 * m + 1]);
        const float2 Ev = cadd(ya, ym);
        const float2 O = cmulc(wsplit[k], csub(ya, ym));
        v[m] = conjf2(cadd(Ev, mul_pi(O)));
        mir[m] = conjf2(cadd(conjf2(Ev), mul_pi(conjf2(O))));
    }
    float2 got[E / 2];
#pragma unroll
    for (int m = 0; m < E / 2; ++m) {
        got[m].x = __shfl_xor_sync(0xffffffffu, mir[m].x, 16);
        got[m].y = __shfl_xor_sync(0xffffffffu, mir[m].y, 16);
    }
    if (i == 0) {
#pragma unroll
        for (int m = 1; m < E / 2; ++m) v[E - m] = mir[m];
    } else if (i == T / 2) {
#pragma unroll
        for (int m = 0; m < E / 2; ++m) v[E - 1 - m] = mir[m];
    } else {
#pragma unroll
        for (int m = 0; m < E / 2; ++m) v[E - 1 - m] = got[m];
    }
}

template <int M, int E, int NB>
__device__ __forceinline__ void irfft_paired(float2 (&v)[E], const float2 (&P)[E], Exch<NB>& ex,
                                             const float2* __restrict__ tw, int t, int i) {
    static_assert(PairedSplit<M, E>::ok, "paired split needs M = E^k");
    using Pl = FftPlan<M, E>;
    paired_unsplit<M, E>(v, P, tw, i);
    {
        float2* b = ex.begin();
        fft_pass<M, E, Pl::radix(0), 1, false>(v, b, tw, i);
        __syncthreads();
        load_strided<M, E>(v, b, t);
        ex.end();
    }
    fft_from_x<M, E, 1, NB>(v, ex, tw, t);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = conjf2(v[s]);
}

}  // namespace rsim
