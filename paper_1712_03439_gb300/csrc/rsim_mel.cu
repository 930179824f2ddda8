// Log-Mel front end (Sec. 3): stacked log-Mel features of one microphone of
// the mixed output.
//
// One warp per frame.  The 512 windowed samples are read as 256 complex
// values z[m] = x[2m] + i x[2m+1] (lane l holds m = l + 32 n for n < 8), and
// the 256-point FFT is done in four steps: an 8-point FFT in registers over n,
// a twiddle exp(-2 pi i l k1 / 256), and for each k1 a 32-point FFT across the
// lanes by five butterfly stages on warp shuffles; lane l then holds
// Z[k1 + 8 rev5(l)].  Z goes through the warp's shared-memory slot for the
// real split (bins k and 256 - k), the power spectrum stays there, and each
// lane sums the triangular Mel filters j = l, l + 32, ... over their bins,
// takes the log and writes the value into every stacked row the frame
// belongs to.  A block is eight warps over kMelFrames consecutive frames of
// one utterance; the window and the twiddles are tabulated per block and the
// filters' nonzero weights (computed on the host) are copied from the launch
// parameters.
#include <cstdint>

#include "rsim_internal.cuh"
#include "rsim_mel.cuh"

namespace rsim {
namespace {

constexpr int kMelWarps = 8;
constexpr int kMelThreads = 32 * kMelWarps;
constexpr int kZPad = 256 + 16;      // Z slot, entry k at k + (k >> 4): the bit-reversed scatter
                                     // and the split's reads meet few bank conflicts

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// exp(-i pi x)
__device__ __forceinline__ float2 expmpi(float x) {
    float s, c;
    sincospif(-x, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ int zslot(int k) { return k + (k >> 4); }

// row offsets (exclusive prefix sum of the rows per utterance), one block
__global__ void __launch_bounds__(1024) k_mel_rows(int32_t U, const int64_t* __restrict__ n_y, MelParams p,
                                                    int64_t* __restrict__ row_off) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (U + 1023) / 1024;
    const int u0 = min(U, t * per), u1 = min(U, u0 + per);
    int64_t sum = 0;
    for (int u = u0; u < u1; ++u) {
        int64_t r, f;
        mel_shape(n_y[u], p, &r, &f);
        sum += r;
    }
    part[t] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;   // exclusive
    for (int u = u0; u < u1; ++u) {
        row_off[u] = run;
        int64_t r, f;
        mel_shape(n_y[u], p, &r, &f);
        run += r;
    }
    if (t == 1023) row_off[U] = part[1023];
}

// grid: (frame chunks of kMelFrames, utterances)
__global__ void __launch_bounds__(kMelThreads, 3)
k_log_mel(const float* __restrict__ y, const int64_t* __restrict__ yoff, const int64_t* __restrict__ n_y, int32_t ch,
          const MelParams p, const int64_t* __restrict__ row_off, float* __restrict__ out) {
    // per-lane tables, indexed so that the lanes of a warp read consecutive entries
    __shared__ float2 winp[kMelFft / 2];       // Hann window pairs (w[2i], w[2i+1])
    __shared__ float2 w512[kMelFft / 2];       // exp(-2 pi i k / 512), the real split
    __shared__ float2 tw1[8][32];              // exp(-2 pi i lane k1 / 256)
    __shared__ float2 twx[4][32];              // cross-lane stage s: the upper lane's twiddle, else 1
    __shared__ float wts[kMelMaxWeights];
    __shared__ int16_t woff[kMelMaxMels + 1], wfirst[kMelMaxMels];
    __shared__ float2 zs[kMelWarps][kZPad];
    __shared__ float ps[kMelWarps][kMelFft / 2 + 1];
    const int u = blockIdx.y;
    const int64_t n = n_y[u];
    int64_t rows64, frames64;
    mel_shape(n, p, &rows64, &frames64);
    const int f0 = blockIdx.x * kMelFrames;
    if (f0 >= frames64) return;
    const int rows = (int)rows64, frames = (int)frames64;   // below 2^31 (checked on the host)
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float* x = y + yoff[u] + (int64_t)ch * n;
    float* o = out + row_off[u] * (int64_t)p.stack * p.n_mels;
    const int width = p.stack * p.n_mels;

    // periodic Hann window, twiddles, and the filter weights from the launch parameters
    for (int k = t; k < kMelFft / 2; k += kMelThreads) {
        winp[k] = make_float2(0.5f - 0.5f * cospif((float)(2 * k) / (kMelFft / 2)),
                              0.5f - 0.5f * cospif((float)(2 * k + 1) / (kMelFft / 2)));
        w512[k] = expmpi((float)k / (kMelFft / 2));
    }
    for (int k = t; k < 8 * 32; k += kMelThreads) tw1[k >> 5][k & 31] = expmpi((float)((k & 31) * (k >> 5)) / 128.f);
    if (t < 4 * 32) {
        const int st = t >> 5, l = t & 31, h = 16 >> st;
        twx[st][l] = (l & h) ? expmpi((float)(l & (h - 1)) / (float)h) : make_float2(1.f, 0.f);
    }
    for (int k = t; k < p.off[p.n_mels]; k += kMelThreads) wts[k] = p.w[k];
    for (int k = t; k <= p.n_mels; k += kMelThreads) woff[k] = p.off[k];
    for (int k = t; k < p.n_mels; k += kMelThreads) wfirst[k] = p.first[k];
    const int rev = __brev(lane) >> 27;
    __syncthreads();

    const int f_end = min(frames, f0 + kMelFrames);
    for (int f = f0 + warp; f < f_end; f += kMelWarps) {
        const float* xf = x + (int64_t)f * p.hop;
        // z[lane + 32 m] for m < 8, windowed
        float2 z[8];
        const bool pairs = (reinterpret_cast<uintptr_t>(xf) & 7) == 0;   // uniform across the warp
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int s = 2 * (lane + 32 * m);
            const float2 wv = winp[lane + 32 * m];
            const float2 xv = pairs ? __ldg(reinterpret_cast<const float2*>(xf + s))
                                    : make_float2(__ldg(xf + s), __ldg(xf + s + 1));
            z[m] = make_float2(xv.x * wv.x, xv.y * wv.y);
        }
        // 8-point FFT over m (decimation in frequency; output index bit-reversed)
        const float r2 = 0.70710678118654752f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float2 a = z[m], b = z[m + 4];
            z[m] = cadd(a, b);
            const float2 d = csub(a, b);
            z[m + 4] = m == 0 ? d
                     : m == 1 ? make_float2(r2 * (d.x + d.y), r2 * (d.y - d.x))
                     : m == 2 ? make_float2(d.y, -d.x)
                              : make_float2(r2 * (d.y - d.x), -r2 * (d.x + d.y));
        }
#pragma unroll
        for (int g = 0; g < 8; g += 4)
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const float2 a = z[g + m], b = z[g + m + 2];
                z[g + m] = cadd(a, b);
                const float2 d = csub(a, b);
                z[g + m + 2] = m == 0 ? d : make_float2(d.y, -d.x);
            }
#pragma unroll
        for (int m = 0; m < 8; m += 2) {
            const float2 a = z[m], b = z[m + 1];
            z[m] = cadd(a, b);
            z[m + 1] = csub(a, b);
        }
        // A[k1] = z[rev3(k1)], times exp(-2 pi i lane k1 / 256)
        float2 A[8];
        A[0] = z[0]; A[1] = z[4]; A[2] = z[2]; A[3] = z[6];
        A[4] = z[1]; A[5] = z[5]; A[6] = z[3]; A[7] = z[7];
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) A[k1] = cmul(A[k1], tw1[k1][lane]);
        // 32-point FFT across the lanes for each k1 (decimation in frequency): the lower lane
        // of a pair keeps a + b, the upper one (b - a) exp(-2 pi i (lane mod h) / 2h)
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int h = 16 >> s;
            const bool upper = lane & h;
            const float sg = upper ? -1.f : 1.f;
            const float2 tw = twx[s < 4 ? s : 0][lane];
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) {
                const float ox = __shfl_xor_sync(0xffffffffu, A[k1].x, h);
                const float oy = __shfl_xor_sync(0xffffffffu, A[k1].y, h);
                const float2 v = make_float2(fmaf(sg, A[k1].x, ox), fmaf(sg, A[k1].y, oy));
                A[k1] = s < 4 ? cmul(v, tw) : v;
            }
        }
        float2* zw = zs[warp];
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) zw[zslot(k1 + 8 * rev)] = A[k1];
        __syncwarp();
        // real split: X[k] = E + exp(-2 pi i k / 512) O, E = (Z[k] + conj Z[256-k]) / 2,
        // O = (Z[k] - conj Z[256-k]) / 2i; power into the warp's slot
        float* pw = ps[warp];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = lane + 32 * q;
            const float2 zk = zw[zslot(k)], zm = zw[zslot((256 - k) & 255)];
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 od = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            const float2 X = cadd(e, cmul(w512[k], od));
            pw[k] = X.x * X.x + X.y * X.y;
        }
        if (lane == 0) {
            const float2 z0 = zw[0];
            const float x256 = z0.x - z0.y;
            pw[256] = x256 * x256;
        }
        __syncwarp();
        // Mel energies, log, and the stacked rows this frame belongs to:
        // rows r with stride r <= f <= stride r + stack - 1, r < rows
        const int r_lo = f >= p.stack ? (f - p.stack) / p.stride + 1 : 0;
        const int r_hi = min(rows - 1, f / p.stride);
        for (int j = lane; j < p.n_mels; j += 32) {
            const int i0 = woff[j], i1 = woff[j + 1];
            const float* pk = pw + wfirst[j] - i0;
            float e = 0.f;
            for (int i = i0; i < i1; ++i) e = fmaf(wts[i], pk[i], e);
            const float v = logf(e + p.floor_);
            for (int r = r_lo; r <= r_hi; ++r)
                o[(int64_t)r * width + (f - r * p.stride) * p.n_mels + j] = v;
        }
        __syncwarp();   // the slots are reused by the warp's next frame
    }
}

}  // namespace

void launch_log_mel(int32_t U, int64_t frames_max, const float* y, const int64_t* yoff, const int64_t* n_y,
                    int32_t ch, const MelParams& p, int64_t* row_off, float* out, cudaStream_t st) {
    k_mel_rows<<<1, 1024, 0, st>>>(U, n_y, p, row_off);
    const int64_t chunks = (frames_max + kMelFrames - 1) / kMelFrames;
    if (chunks > 0 && U > 0)
        k_log_mel<<<dim3((unsigned)chunks, (unsigned)U), kMelThreads, 0, st>>>(y, yoff, n_y, ch, p, row_off, out);
}

}  // namespace rsim
