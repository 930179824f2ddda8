// Image-method room impulse responses (Eq. 1, Sec. 2).
//
// A block owns one window of kImgWindow taps of one RIR and accumulates it in
// shared memory: each thread takes (a, b) pairs of virtual-room indices and
// walks the 2K+1 rooms c of each pair, landing every image whose delay falls
// inside the window with a shared-memory atomic add; the block then writes
// the window out whole (zeros included) with 16-byte stores, so the output is
// written once and never read.  The per-axis squared offsets and reflection
// powers of the 2K+1 virtual rooms are tabulated per block and a pair's x + y
// part is held in registers, which leaves per image one addition, a square
// root and a multiply for the delay and two multiplies and a reciprocal square
// root for the amplitude.  Work per image does not depend on the RIR length, so
// the window is as large as static shared memory allows (44 KB; four blocks of
// ten warps fit on an SM) and covers most RIRs in one pass.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "rsim.h"
#include "rsim_internal.cuh"

namespace rsim {
namespace {

constexpr int kImgThreads = 320;                  // ten warps: the paper's 17 x 17 (a, b) pairs in one round
constexpr int kImgWindow = 11264;                 // taps per shared-memory window
constexpr int kImgMaxOrder = 32;
constexpr int kImgMaxSide = 2 * kImgMaxOrder + 1;  // virtual rooms per axis
constexpr int64_t kImgMaxLen = int64_t(1) << 24;   // taps of one RIR (delays exact in FP32)

enum : int32_t { kImgBadGeom = 1, kImgBadLen = 2 };

// Offset from the microphone coordinate m to the image coordinate in virtual
// room a along one axis: a*len + s for even a, (a+1)*len - s for odd a; each
// step one correctly rounded FP32 operation (no contraction).
__device__ __forceinline__ float image_offset(int a, float len, float s, float m) {
    const float p = (a & 1) ? __fsub_rn(__fmul_rn((float)(a + 1), len), s)
                            : __fadd_rn(__fmul_rn((float)a, len), s);
    return __fsub_rn(p, m);
}

__device__ __forceinline__ bool geom_valid(const rsim_image_geom& g) {
    bool ok = g.refl >= 0.f && g.refl < 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        ok = ok && g.room[k] > 0.f && isfinite(g.room[k]) && g.src[k] > 0.f && g.src[k] < g.room[k] &&
             g.mic[k] > 0.f && g.mic[k] < g.room[k];
    return ok;
}

// Per axis and virtual-room index a - K: (squared offset to the microphone, r^|a - K|),
// built by the block's first 3 (2K + 1) threads (the caller synchronises).
__device__ __forceinline__ void image_tables(const rsim_image_geom& g, int K, float2 (*tab)[kImgMaxSide]) {
    const int t = threadIdx.x;
    const int S = 2 * K + 1;
    if (t < 3 * S) {
        const int k = t / S, ai = t - k * S;
        // axis k picked by selects (a runtime index into g would go through local memory)
        const float len = k == 0 ? g.room[0] : k == 1 ? g.room[1] : g.room[2];
        const float s = k == 0 ? g.src[0] : k == 1 ? g.src[1] : g.src[2];
        const float m = k == 0 ? g.mic[0] : k == 1 ? g.mic[1] : g.mic[2];
        const float e = image_offset(ai - K, len, s, m);
        // r^|a| by repeated squaring
        float p = 1.f, b = g.refl;
        for (int q = abs(ai - K); q; q >>= 1) {
            if (q & 1) p *= b;
            b *= b;
        }
        tab[k][ai] = make_float2(__fmul_rn(e, e), p);
    }
}

// Lands every image whose delay falls in [w0, w0 + wl) at win[delay - w0 + lead]
// (shared memory, zeroed by the caller) with shared-memory atomics; threads take
// (a, b) pairs of virtual rooms and walk the rooms c.  Returns true in a thread
// that met an image at distance zero (the caller combines them).
__device__ __forceinline__ bool land_images(const float2 (*tab)[kImgMaxSide], int K, float rate, int64_t w0,
                                            int wl, int lead, float* win) {
    const int S = 2 * K + 1;
    const int P = S * S;
    const float w0_f = (float)w0;
    bool at_mic = false;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int ai = p / S, bi = p - ai * S;
        const float2 ta = tab[0][ai], tb = tab[1][bi];
        const float sab = __fadd_rn(ta.x, tb.x);   // (x^2 + y^2) + z^2, in that order
        const float rab = ta.y * tb.y;
#pragma unroll 4
        for (int ci = 0; ci < S; ++ci) {
            const float2 tc = tab[2][ci];
            const float d2 = __fadd_rn(sab, tc.x);
            at_mic |= !(d2 > 0.f);   // an image at the microphone
            // delay = ceil(d * rate); ceil and w0 are integers, exact below 2^24, so the
            // offset is exact wherever it can land in the window (wl <= nh - w0)
            const int i = __float2int_rz(ceilf(__fmul_rn(__fsqrt_rn(d2), rate)) - w0_f);
            if ((unsigned)i < (unsigned)wl) atomicAdd(&win[i + lead], rab * tc.y * rsqrtf(d2));
        }
    }
    return at_mic;
}

// grid: R * nw blocks; block b takes RIR b / nw and windows b % nw, b % nw + nw, ...
__global__ void __launch_bounds__(kImgThreads, 4)
k_image_rirs(int32_t R, int32_t nw, const rsim_image_geom* __restrict__ geom,
             const int64_t* __restrict__ off, int32_t K, float fs, float c0, float* __restrict__ rir,
             int32_t* status) {
    // tap n of the window sits at win[n + lead], lead = the output's offset from a
    // 16-byte boundary, so that 16-byte chunks of win map onto 16-byte chunks of rir
    __shared__ __align__(16) float win[kImgWindow + 4];
    // per axis and virtual-room index: (squared offset, r^|index|)
    __shared__ float2 tab[3][kImgMaxSide];
    const int t = threadIdx.x;
    const int r = (int)(blockIdx.x / (unsigned)nw);
    const int w_first = (int)(blockIdx.x % (unsigned)nw);
    if (r >= R) return;
    const int64_t o0 = off[r];
    const int64_t nh = off[r + 1] - o0;
    if (nh < 0 || nh > kImgMaxLen) {
        if (t == 0 && w_first == 0 && status) atomicOr(status, kImgBadLen);
        return;
    }
    if ((int64_t)w_first * kImgWindow >= nh) return;
    const rsim_image_geom g = geom[r];
    const bool valid = geom_valid(g);
    image_tables(g, K, tab);
    // samples per metre, one rounding (the same value on every side of the comparison)
    const float rate = __fdiv_rn(fs, c0);
    float4* win4 = reinterpret_cast<float4*>(win);
    for (int64_t w = w_first; w * kImgWindow < nh; w += nw) {
        const int64_t w0 = w * kImgWindow;
        const int wl = (int)(nh - w0 < kImgWindow ? nh - w0 : (int64_t)kImgWindow);
        float* dst = rir + o0 + w0;
        const int lead = (int)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3);
        for (int q = t; q < (kImgWindow + 4) / 4; q += kImgThreads) win4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();   // also publishes the tables on the first pass
        const bool at_mic = land_images(tab, K, rate, w0, wl, lead, win);
        const bool bad = __syncthreads_or(at_mic) || !valid;
        if (bad && t == 0 && w == w_first && status) atomicOr(status, kImgBadGeom);
        // 16-byte chunks of win [4q, 4q + 4) hold taps 4q - lead .. 4q + 3 - lead; the first
        // and last chunk may be partial
        float* dsta = dst - lead;   // 16-byte aligned; its first `lead` floats are not ours
        const int end = lead + wl;
        for (int q = t; 4 * q < end; q += kImgThreads) {
            const int lo = 4 * q;
            float4 v = bad ? make_float4(0.f, 0.f, 0.f, 0.f) : win4[q];
            if (lo >= lead && lo + 4 <= end) {
                *reinterpret_cast<float4*>(dsta + lo) = v;
            } else {
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (lo + k >= lead && lo + k < end) dsta[lo + k] = e[k];
            }
        }
        __syncthreads();   // the window is reused by the next pass
    }
}

// K1 fused with Eq. 1, for plans fed by room geometry (rsim_filter_mix_rooms): one
// block per RIR (grid-stride) lands every image of the RIR in shared memory (the
// whole RIR, Nh_max floats of dynamic shared memory), takes the cut-off there with
// the same decision as the standalone scan (cut_rir), and writes only the kept taps
// [0, L) to `kept` (plan scratch in the packed RIR layout, read by the spectrum
// kernel); with `full` non-NULL every tap also goes there.  An invalid geometry or
// an image at the microphone gives an all-zero RIR (L = 1) and latches
// kErrBadGeometry.
constexpr int kCutThreads = 320;

__global__ void __launch_bounds__(kCutThreads)
k_image_cut(DevBatch B, const rsim_image_geom* __restrict__ geom, int32_t K, float fs, float c0, double factor,
            float sqrt_factor, int none, float* __restrict__ kept, float* __restrict__ full,
            float* __restrict__ ekf) {
    extern __shared__ __align__(16) float hwin[];
    __shared__ float2 tab[3][kImgMaxSide];
    __shared__ CutScratch cs;
    const int t = threadIdx.x;
    const float rate = __fdiv_rn(fs, c0);
    for (int r = blockIdx.x; r < B.R; r += gridDim.x) {
        const int nh = B.rir_len[r];
        const int64_t o0 = B.roff[r];
        const rsim_image_geom g = geom[r];
        const bool valid = geom_valid(g);
        __syncthreads();                         // the previous RIR's readers are done
        image_tables(g, K, tab);
        for (int i = t; i < nh; i += kCutThreads) hwin[i] = 0.f;
        __syncthreads();
        const bool at_mic = land_images(tab, K, rate, 0, nh, 0, hwin);
        if (__syncthreads_or(at_mic) || !valid) {
            for (int i = t; i < nh; i += kCutThreads) hwin[i] = 0.f;
            if (t == 0) atomicOr(B.err, kErrBadGeometry);
            __syncthreads();
        }
        float frac = 1.f;
        const int L = cut_rir([&](int i) { return hwin[i]; }, nh, factor, sqrt_factor, none, ekf != nullptr, &frac,
                              cs);
        for (int i = t; i < L; i += kCutThreads) kept[o0 + i] = hwin[i];
        if (full)
            for (int i = t; i < nh; i += kCutThreads) full[o0 + i] = hwin[i];
        if (t == 0) {
            B.L[r] = L;
            if (ekf) ekf[r] = frac;
        }
    }
}

}  // namespace

int image_cut_smem(int nh_max) { return (int)sizeof(float) * std::max(nh_max, 1); }

int image_cut_grid(int nh_max, int R, int sms) {
    const int smem = image_cut_smem(nh_max);
    cudaFuncSetAttribute(k_image_cut, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_image_cut, kCutThreads, smem);
    return std::max(1, std::min(R, std::max(occ, 1) * std::max(sms, 1)));
}

void launch_image_cut(const DevBatch& B, const rsim_image_geom* geom, int K, float fs, float c0, double factor,
                      int none, int nh_max, float* kept, float* full, float* ekf, int grid, cudaStream_t st) {
    k_image_cut<<<grid, kCutThreads, image_cut_smem(nh_max), st>>>(B, geom, K, fs, c0, factor,
                                                                   (float)std::sqrt(factor), none, kept, full, ekf);
}

}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_image_rirs(void* stream, int32_t num_rirs, const rsim_image_geom* geom,
                                       const int64_t* rir_off, int64_t max_len, int32_t order, float fs,
                                       float c0, float* rir, int32_t* status) {
    if (num_rirs < 0 || order < 0 || order > kImgMaxOrder || !(fs > 0.f) || !(c0 > 0.f) ||
        !std::isfinite(fs) || !std::isfinite(c0) || max_len < 0 || max_len > kImgMaxLen) {
        set_last_error("rsim_image_rirs: need num_rirs >= 0, order in [0, 32], finite fs, c0 > 0, "
                       "max_len in [0, 2^24]");
        return RSIM_E_INVALID;
    }
    if (num_rirs > 0 && (!geom || !rir_off || !rir)) {
        set_last_error("rsim_image_rirs: null geometry, offset or output pointer");
        return RSIM_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (status) e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) {
        set_last_error((std::string("rsim_image_rirs: cudaMemsetAsync: ") + cudaGetErrorString(e)).c_str());
        return RSIM_E_CUDA;
    }
    if (num_rirs == 0) return RSIM_OK;
    const int64_t nw = std::max<int64_t>(1, (max_len + kImgWindow - 1) / kImgWindow);
    const int64_t blocks = (int64_t)num_rirs * nw;
    if (blocks > 0x7fffffff) {
        set_last_error("rsim_image_rirs: too many RIR windows for one launch; split the batch");
        return RSIM_E_INVALID;
    }
    k_image_rirs<<<(unsigned)blocks, kImgThreads, 0, st>>>(num_rirs, (int32_t)nw, geom, rir_off, order, fs,
                                                          c0, rir, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error((std::string("rsim_image_rirs launch: ") + cudaGetErrorString(e)).c_str());
        return RSIM_E_CUDA;
    }
    return RSIM_OK;
}
