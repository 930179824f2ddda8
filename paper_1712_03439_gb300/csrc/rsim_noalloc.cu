// Allocation-free gains entry point.
//
// Some callers cannot allocate device memory at the point where they need
// the per-source gains: code running under a memory manager that owns every
// device allocation (a framework's caching allocator, a real-time audio
// engine that pre-reserves its memory at start-up), or code where an
// allocation would stall the device at the wrong moment.  A plan allocates
// its scratch in rsim_plan, so those callers cannot use one.
// rsim_source_gains_noalloc computes the same gains as rsim_filter_mix with
// gain_mode = 0, using the library's source-power kernel, but its scratch
// (per-chunk partial sums and the batch offsets) lives in the fixed
// file-scope device array below instead of plan memory.
#include "rsim.h"
#include "rsim_internal.cuh"

#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

namespace rsim {

// The scratch of every call: 2 MiB, reserved on each GPU that loads the
// library for as long as the library stays loaded.
constexpr size_t kNoAllocScratchBytes = 2u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
void* g_na_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name only stands in for the symbol; the address the kernels
// need comes from cudaGetSymbolAddress, taken once per device with that
// device current.
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Offsets of the packed sources (one thread; the batch is small by the
// scratch bound): src0[u] = first source of utterance u, xoff[s] = offset of
// source s in x, src_utt[s] = utterance of source s.
__global__ void k_offsets_noalloc(int U, const int32_t* __restrict__ nsrc, const int64_t* __restrict__ nx,
                                  int32_t* __restrict__ src0, int64_t* __restrict__ xoff,
                                  int32_t* __restrict__ src_utt) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int32_t s = 0;
    int64_t o = 0;
    for (int u = 0; u < U; ++u) {
        src0[u] = s;
        for (int i = 0; i < nsrc[u]; ++i) {
            src_utt[s] = u;
            xoff[s++] = o;
            o += nx[u];
        }
    }
    src0[U] = s;
    xoff[s] = o;
}

// alpha_0 = 1, alpha_i = sqrt(P_0 / P_i 10^(-SNR_i/10)) from the partial
// sums, added in chunk order as the planner does; a silent noise source
// gets NaN (no finite gain meets its SNR).
__global__ void k_gains_noalloc(DevBatch B, const float* __restrict__ snr_db, float* __restrict__ gains) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.U) return;
    const int s0 = B.src0[u], I = B.src0[u + 1] - B.src0[u];
    const double nx = (double)B.n_x[u];
    const int nch = (int)((B.n_x[u] + kPowerChunk - 1) / kPowerChunk);
    double P0 = 0.0;
    for (int c = 0; c < nch; ++c) P0 += B.pow_part[(int64_t)s0 * B.CH + c];
    P0 /= nx;
    gains[s0] = 1.f;
    for (int i = 1; i < I; ++i) {
        double Pi = 0.0;
        for (int c = 0; c < nch; ++c) Pi += B.pow_part[(int64_t)(s0 + i) * B.CH + c];
        Pi /= nx;
        gains[s0 + i] = (Pi > 0.0) ? (float)sqrt(P0 / Pi * pow(10.0, -(double)snr_db[s0 + i] / 10.0))
                                   : __int_as_float(0x7fc00000);
    }
}

}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_source_gains_noalloc(void* stream, int32_t num_utts, const int32_t* num_sources,
                                                 const int64_t* num_samples, const float* x,
                                                 const float* snr_db, float* gains) {
    if (num_utts < 1 || !num_sources || !num_samples || !x || !snr_db || !gains) {
        set_last_error("rsim_source_gains_noalloc: bad argument");
        return RSIM_E_INVALID;
    }
    const int U = num_utts;
    int64_t S = 0, nx_max = 1;
    for (int u = 0; u < U; ++u) {
        if (num_sources[u] < 1 || num_sources[u] > kMaxSources || num_samples[u] < 1) {
            set_last_error("rsim_source_gains_noalloc: num_sources must be in [1, 16], num_samples >= 1");
            return RSIM_E_INVALID;
        }
        S += num_sources[u];
        nx_max = std::max<int64_t>(nx_max, num_samples[u]);
    }
    const int64_t CH = (nx_max + kPowerChunk - 1) / kPowerChunk;
    // scratch layout: num_sources [U] i32 | n_x [U] i64 | src0 [U+1] i32 |
    //                 xoff [S+1] i64 | src_utt [S] i32 | partial sums [S*CH] f64
    const size_t o_nsrc = 0;
    const size_t o_nx = align256(o_nsrc + sizeof(int32_t) * U);
    const size_t o_src0 = align256(o_nx + sizeof(int64_t) * U);
    const size_t o_xoff = align256(o_src0 + sizeof(int32_t) * (U + 1));
    const size_t o_sutt = align256(o_xoff + sizeof(int64_t) * (S + 1));
    const size_t o_part = align256(o_sutt + sizeof(int32_t) * S);
    const size_t need = o_part + sizeof(double) * (size_t)S * (size_t)CH;
    if (need > kNoAllocScratchBytes) {
        set_last_error(("rsim_source_gains_noalloc: this batch needs " + std::to_string(need) +
                        " bytes of scratch but the fixed maximum is " +
                        std::to_string(kNoAllocScratchBytes) + "; split the batch").c_str());
        return RSIM_E_UNSUPPORTED;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error("rsim_source_gains_noalloc: no usable current device");
        return RSIM_E_CUDA;
    }
    void* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) {
        set_last_error((std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        return RSIM_E_CUDA;
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream;
    // the caller's host shape arrays go straight into the scratch
    e = cudaMemcpyAsync(b + o_nsrc, num_sources, sizeof(int32_t) * U, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_nx, num_samples, sizeof(int64_t) * U, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        set_last_error((std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e)).c_str());
        return RSIM_E_CUDA;
    }
    DevBatch B{};
    B.U = U;
    B.S = (int32_t)S;
    B.CH = (int32_t)CH;
    B.n_src = reinterpret_cast<const int32_t*>(b + o_nsrc);
    B.n_x = reinterpret_cast<const int64_t*>(b + o_nx);
    B.src0 = reinterpret_cast<const int32_t*>(b + o_src0);
    B.xoff = reinterpret_cast<const int64_t*>(b + o_xoff);
    B.src_utt = reinterpret_cast<const int32_t*>(b + o_sutt);
    B.pow_part = reinterpret_cast<double*>(b + o_part);
    k_offsets_noalloc<<<1, 32, 0, st>>>(U, B.n_src, B.n_x, reinterpret_cast<int32_t*>(b + o_src0),
                                        reinterpret_cast<int64_t*>(b + o_xoff),
                                        reinterpret_cast<int32_t*>(b + o_sutt));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(S * CH, (int64_t)std::max(sms, 1) * 8));
    launch_power(B, x, grid, st);
    k_gains_noalloc<<<(U + 255) / 256, 256, 0, st>>>(B, snr_db, gains);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error((std::string("rsim_source_gains_noalloc launch: ") + cudaGetErrorString(e)).c_str());
        return RSIM_E_CUDA;
    }
    return RSIM_OK;
}
