// Image-method room impulse responses (Eq. 1, Sec. 2).
//
// A block owns one window of kImgWindow taps of one RIR and accumulates it in
// shared memory: every thread walks its share of the (2K+1)^3 images, lands
// each one whose delay falls inside the window with a shared-memory atomic
// add, and the block then writes the window out whole (zeros included), so
// the output is written once and never read.  The per-axis squared offsets of
// the 2K+1 virtual rooms and the powers r^g are tabulated per block, which
// leaves two additions, a square root, a multiply and a division per image.
// Work per image is independent of the RIR length, so the window is as large
// as static shared memory allows (44 KB; five blocks fit on an SM), which
// covers most RIRs in one pass.
#include <algorithm>
#include <cmath>
#include <string>

#include "rsim.h"
#include "rsim_internal.cuh"

namespace rsim {
namespace {

constexpr int kImgThreads = 256;
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

// grid: R * nw blocks; block b takes RIR b / nw and windows b % nw, b % nw + nw, ...
__global__ void __launch_bounds__(kImgThreads)
k_image_rirs(int32_t R, int32_t nw, const rsim_image_geom* __restrict__ geom,
             const int64_t* __restrict__ off, int32_t K, float fs, float c0, float* __restrict__ rir,
             int32_t* status) {
    __shared__ float win[kImgWindow];
    __shared__ float sq[3][kImgMaxSide];             // squared offset per axis and room index
    __shared__ float pw[3 * kImgMaxOrder + 1];       // r^g
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
    const int S = 2 * K + 1;
    const int V = S * S * S;
    if (t < 3 * S) {
        const int k = t / S, ai = t - k * S;
        // axis k picked by selects (a runtime index into g would go through local memory)
        const float len = k == 0 ? g.room[0] : k == 1 ? g.room[1] : g.room[2];
        const float s = k == 0 ? g.src[0] : k == 1 ? g.src[1] : g.src[2];
        const float m = k == 0 ? g.mic[0] : k == 1 ? g.mic[1] : g.mic[2];
        const float e = image_offset(ai - K, len, s, m);
        sq[k][ai] = __fmul_rn(e, e);
    }
    if (t <= 3 * K) {
        // r^t by repeated squaring
        float p = 1.f, b = g.refl;
        for (int e = t; e; e >>= 1) {
            if (e & 1) p *= b;
            b *= b;
        }
        pw[t] = p;
    }
    // digits (base S) of the thread's first image and of the stride between its images
    const int c_first = t % S, b_first = (t / S) % S, a_first = t / (S * S);
    const int dc = kImgThreads % S, db = (kImgThreads / S) % S, da = kImgThreads / (S * S);
    const float nh_f = (float)nh;
    for (int64_t w = w_first; w * kImgWindow < nh; w += nw) {
        const int64_t w0 = w * kImgWindow;
        const int wl = (int)(nh - w0 < kImgWindow ? nh - w0 : (int64_t)kImgWindow);
        const float w0_f = (float)w0, wl_f = (float)wl;
        for (int n = t; n < wl; n += kImgThreads) win[n] = 0.f;
        __syncthreads();   // also publishes sq and pw on the first pass
        bool at_mic = false;
        int ai = a_first, bi = b_first, ci = c_first;
        for (int v = t; v < V; v += kImgThreads) {
            const float d2 = __fadd_rn(__fadd_rn(sq[0][ai], sq[1][bi]), sq[2][ci]);
            if (d2 > 0.f) {
                const float d = __fsqrt_rn(d2);
                const float n_f = ceilf(__fdiv_rn(__fmul_rn(d, fs), c0));
                // n_f and w0 are integers below 2^24 here, so n_f - w0 is exact
                if (n_f < nh_f && n_f >= w0_f && n_f - w0_f < wl_f) {
                    const int gv = abs(ai - K) + abs(bi - K) + abs(ci - K);
                    atomicAdd(&win[(int)(n_f - w0_f)], __fdiv_rn(pw[gv], d));
                }
            } else {
                at_mic = true;
            }
            // next image of this thread: v + kImgThreads in base S
            ci += dc;
            if (ci >= S) { ci -= S; ++bi; }
            bi += db;
            if (bi >= S) { bi -= S; ++ai; }
            ai += da;
        }
        const bool bad = __syncthreads_or(at_mic) || !valid;
        if (bad && t == 0 && w == w_first && status) atomicOr(status, kImgBadGeom);
        float* dst = rir + o0 + w0;
        for (int n = t; n < wl; n += kImgThreads) dst[n] = bad ? 0.f : win[n];
        __syncthreads();   // the window is reused by the next pass
    }
}

}  // namespace
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
