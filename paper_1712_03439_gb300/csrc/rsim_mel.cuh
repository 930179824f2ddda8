// Declarations of the log-Mel front end shared by its kernels and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsim {

// log-Mel front end (Sec. 3): frames of kMelFft samples every hop samples,
// n_mels triangular filters, ln(E + floor), stack frames per row, rows every
// stride frames
constexpr int kMelFft = 512;
constexpr int kMelMaxMels = 128;
constexpr int kMelFrames = 64;      // frames per block
constexpr int kMelMaxWeights = 2 * (kMelFft / 2 + 1);   // a bin lies inside at most two triangles
struct MelParams {
    int32_t hop, n_mels, stack, stride;
    float floor_;                      // added to each filter energy before the log
    // filter j's nonzero weights w[off[j] .. off[j+1]) on bins first[j], first[j] + 1, ...
    // (computed in FP64 on the host, rounded once)
    int16_t off[kMelMaxMels + 1];
    int16_t first[kMelMaxMels];
    float w[kMelMaxWeights];
};
// rows of stacked features and the frames they need, from n samples
__host__ __device__ inline void mel_shape(int64_t n, const MelParams& p, int64_t* rows, int64_t* frames) {
    const int64_t T = n >= kMelFft ? (n - kMelFft) / p.hop + 1 : 0;
    const int64_t R = T >= p.stack ? (T - p.stack) / p.stride + 1 : 0;
    *rows = R;
    *frames = R ? (R - 1) * p.stride + p.stack : 0;
}
void launch_log_mel(int32_t U, int64_t frames_max, const float* y, const int64_t* yoff, const int64_t* n_y,
                    int32_t ch, const MelParams& p, int64_t* row_off, float* out, cudaStream_t st);

}  // namespace rsim
