// C-ABI of the room-simulator filter-and-mix library: plan creation, scratch
// management, twiddle tables and the launch sequences of the forward and
// backward passes.  Every step of the computation runs in the kernels of
// rsim_prep.cu, rsim_forward.cu and rsim_backward.cu.
#include "rsim.h"
#include "rsim_fft.cuh"
#include "rsim_internal.cuh"
#include "rsim_mel.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace rsim;

namespace {

thread_local std::string g_err;

rsim_status fail(rsim_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

rsim_status cuda_fail(cudaError_t e, const char* what) {
    return fail(RSIM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev_); }
  private:
    int prev_ = 0;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// exp(-2 pi i num / den) in FP64, rounded once to FP32
float2 twiddle(int64_t num, int64_t den) {
    num %= den;
    const double ang = -2.0 * M_PI * (double)num / (double)den;
    return make_float2((float)std::cos(ang), (float)std::sin(ang));
}

template <int M, int E>
std::vector<float2> twiddle_table() {
    using P = FftPlan<M, E>;
    std::vector<float2> tw(P::TW_LEN);
    // pass p >= 1: rows w^(2^j), j < log2(radix), of lp(p) entries each
    for (int p = 1; p < P::NPASS; ++p) {
        const int R = P::radix(p), LP = P::lp(p);
        for (int j = 0; j < ilog2(R); ++j)
            for (int k = 0; k < LP; ++k)
                tw[P::tw_off(p) + j * LP + k] = twiddle((int64_t)(1 << j) * k, (int64_t)LP * R);
    }
    for (int k = 0; k <= M / 2; ++k) tw[P::OFF_SPLIT + k] = twiddle(k, 2 * M);
    return tw;
}

std::vector<float2> twiddle_table_for(int logN, int E) {
    switch (logN * 100 + E) {
        case 1108: return twiddle_table<1024, 8>();
        case 1116: return twiddle_table<1024, 16>();
        case 1208: return twiddle_table<2048, 8>();
        case 1216: return twiddle_table<2048, 16>();
        case 1308: return twiddle_table<4096, 8>();
        case 1316: return twiddle_table<4096, 16>();
        case 1408: return twiddle_table<8192, 8>();
        case 1416: return twiddle_table<8192, 16>();
    }
    return {};
}

}  // namespace

constexpr int kRing = 64;

// Captured launch sequences, one per set of buffer pointers (a few sets, so
// callers that alternate buffers -- double-buffered copies -- replay instead of
// re-capturing); the least recently used one is replaced.
constexpr int kGraphSlots = 4;
struct GraphCache {
    const void* key[kGraphSlots][8] = {};
    cudaGraphExec_t exec[kGraphSlots] = {};
    uint64_t used[kGraphSlots] = {};
    uint64_t tick = 0;
    void destroy() {
        for (int s = 0; s < kGraphSlots; ++s)
            if (exec[s]) {
                cudaGraphExecDestroy(exec[s]);
                exec[s] = nullptr;
            }
    }
};

struct StageTimer {
    bool on = false;
    int count[RSIM_NUM_STAGES] = {};
    cudaEvent_t ev[RSIM_NUM_STAGES][kRing][2] = {};
};

struct rsim_plan_s {
    int device = 0;
    int sms = 0;
    DevBatch B{};
    Queues Q{};
    double factor = 0.0;
    int none = 0;
    int gain_mode = 0;
    int mask = 0;
    void* dmem = nullptr;
    size_t dbytes = 0;
    float2* Hc = nullptr;
    float* tails = nullptr;
    float* dhp = nullptr;
    float* dap = nullptr;
    Twiddles tw[kNumBuckets] = {};
    int grid_trunc = 1, grid_pow = 1;
    int grid_spec[kNumBuckets] = {}, grid_fwd[kNumBuckets] = {}, grid_bwd[kNumBuckets] = {};
    bool fwd_done = false;
    StageTimer timer;
    // one stream per FFT size so the per-size launches run side by side
    cudaStream_t bs[kNumBuckets] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kNumBuckets] = {};
    // CUDA graphs of the forward and backward sequences (replayed per call)
    bool use_graphs = true;
    cudaStream_t cap = nullptr;     // capture stream
    cudaStream_t aux = nullptr;     // side stream of the forward's first stage
    cudaEvent_t ev_aux = nullptr;
    cudaEvent_t ev_plan = nullptr;  // the planner done (the backward partition waits for it)
    cudaEvent_t ev_part = nullptr;  // the backward partition done (the forward's end waits for it)
    GraphCache gfwd, gbwd;
    // output samples per microphone of each utterance (host copy) and the row
    // offsets of the log-Mel features (device, written per call)
    std::vector<int64_t> h_ny;
    int64_t* mel_row_off = nullptr;
    // per-(i, j) gains (gain_mode 2): unit source gains for the kernels, and the RIR
    // buffer of the last forward (the backward's gain gradient reads it)
    float* ones = nullptr;
    const float* fwd_rir = nullptr;
    // RIRs from room geometry (rsim_filter_mix_rooms): the kept taps, the launch shape of
    // the fused generation and cut-off, its graphs and the scalar arguments they hold
    float* rir_kept = nullptr;
    int nh_max = 1, grid_cut = 1;
    // the allocation's pieces (bytes each, in carving order): a reshape fits the new
    // shape's pieces into them at the same offsets
    std::vector<size_t> piece_cap;
    rsim_plan_desc desc_fixed{};     // the fields a reshape must keep (pointers cleared)
    GraphCache grooms;
    int32_t rooms_order = -1;
    float rooms_fs = 0.f, rooms_c0 = 0.f;
    // gains from reverberant SNRs (gain_mode 3): a plan over the sources, each its own
    // one-microphone utterance with its RIR to the reference microphone, whose output
    // (laid out like x) feeds the source-power scan; the RIRs are gathered for it
    rsim_plan_t rev = nullptr;
    const int64_t* rev_src_off = nullptr;   // [S] offset of each source's reference RIR in rir
    const int64_t* rev_dst_off = nullptr;   // [S + 1] its offset in rev_rir
    float* rev_rir = nullptr;
    float* rev_y = nullptr;
    // Utterances whose RIRs may reach beyond one block of the largest size: uniformly
    // partitioned convolution.  A plan over those utterances, in which virtual source
    // (i, q) is source i delayed by q * part_len samples and filtered by taps
    // [q * part_len, (q + 1) * part_len) of its RIRs, does the work for the ones the
    // planner sends there (defer); segment copies and sums map x, the RIRs, the gains and
    // grad_y onto it and its outputs and gradients back, for those utterances only.
    rsim_plan_t part = nullptr;
    struct Segs {
        const int64_t *src, *dst, *lead, *copy, *tail;
        const int64_t* utt;               // utterance of the partitioned plan (skip unless deferred)
        const int64_t *lim_r, *lim_off;   // copy at most L[lim_r] - lim_off values (NULL: all)
        int64_t n;
        int64_t out_n;                    // floats of the destination buffer
    };
    struct Sums { const int64_t *out, *len, *t0, *src, *tlen, *utt; int64_t n, out_n; };
    Segs seg_x{}, seg_h{}, seg_a{}, seg_dh{}, seg_y{}, seg_gy{};
    Sums sum_dx{}, sum_da{};
    float *part_x = nullptr, *part_rir = nullptr, *part_a = nullptr, *part_y = nullptr;
    float *part_dx = nullptr, *part_dh = nullptr, *part_da = nullptr;
    uint8_t* defer = nullptr;             // [utterances of the partitioned plan]
    std::vector<int32_t> part_utt;        // its utterance k is utterance part_utt[k] here
    void* part_mem = nullptr;
    size_t part_bytes = 0;
};

namespace {
// segment o of a deferred utterance: lead[o] zeros, then copy[o] values from in + src[o]
// (at most L[lim_r[o]] - lim_off[o] of them: a part of a cut RIR, or of its gradient; zeros
// in place of the rest), then tail[o] zeros, written from out + dst[o]
// (B: the outer plan, whose planner set the deferral flags and whose cut-off set L).
// The blocks of one grid row (blockIdx.y) take segments o = y, y + gridDim.y, ...; the
// gridDim.x blocks of a row split each segment's values between them.
__global__ void k_copy_segs(DevBatch B, rsim_plan_s::Segs g, const float* __restrict__ in, float* __restrict__ out) {
    const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dk = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = blockIdx.y; o < g.n; o += gridDim.y) {
        if (!B.defer[g.utt[o]]) continue;
        float* d = out + g.dst[o];
        const float* s = in + g.src[o];
        const int64_t a = g.lead[o], n = a + g.copy[o] + g.tail[o];
        int64_t c = g.copy[o];
        if (g.lim_r) c = max((int64_t)0, min(c, (int64_t)B.L[g.lim_r[o]] - g.lim_off[o]));
        for (int64_t k = k0; k < n; k += dk)
            if (RSIM_STORE_OK(B, d + k, out, 4 * g.out_n)) d[k] = (k >= a && k < a + c) ? s[k - a] : 0.f;
    }
}

// output o of a deferred utterance, length len[o]: out[out[o] + m] = sum over terms q in
// [t0[o], t0[o + 1]) of in[src[q] + m] for m < tlen[q] (terms added in order)
__global__ void k_sum_segs(DevBatch B, rsim_plan_s::Sums g, const float* __restrict__ in, float* __restrict__ out) {
    const int64_t m0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dm = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = blockIdx.y; o < g.n; o += gridDim.y) {
        if (!B.defer[g.utt[o]]) continue;
        const int64_t q0 = g.t0[o], q1 = g.t0[o + 1];
        for (int64_t m = m0; m < g.len[o]; m += dm) {
            float acc = 0.f;
            for (int64_t q = q0; q < q1; ++q)
                if (m < g.tlen[q]) acc += in[g.src[q] + m];
            if (RSIM_STORE_OK(B, out + g.out[o] + m, out, 4 * g.out_n)) out[g.out[o] + m] = acc;
        }
    }
}

// copies RIR s from rir + src_off[s] to dst + dst_off[s] (dst_off[s + 1] - dst_off[s] taps)
__global__ void k_gather_rirs(int64_t n, const int64_t* __restrict__ src_off, const int64_t* __restrict__ dst_off,
                              const float* __restrict__ rir, float* __restrict__ dst) {
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        const float* a = rir + src_off[s];
        float* b = dst + dst_off[s];
        const int64_t len = dst_off[s + 1] - dst_off[s];
        for (int64_t k = threadIdx.x; k < len; k += blockDim.x) b[k] = a[k];
    }
}
}  // namespace

namespace {

// records the start (end = false) or end of a stage when timing is enabled
void stage_mark(rsim_plan_t p, int stage, bool end, cudaStream_t st) {
    if (!p->timer.on) return;
    const int slot = p->timer.count[stage] % kRing;
    cudaEvent_t& e = p->timer.ev[stage][slot][end ? 1 : 0];
    if (!e) cudaEventCreate(&e);
    cudaEventRecord(e, st);
    if (end) ++p->timer.count[stage];
}

// Runs launch(logN, stream) for every allowed FFT size on that size's own
// stream, forked from and joined back into st.  Largest sizes go first: their
// tiles are the longest.
template <typename F>
void fan_out(rsim_plan_t p, cudaStream_t st, F launch) {
    cudaEventRecord(p->ev_fork, st);
    for (int m = kMaxLog; m >= kMinLog; --m) {
        if (!((p->mask >> m) & 1)) continue;
        const int b = m - kMinLog;
        cudaStreamWaitEvent(p->bs[b], p->ev_fork, 0);
        launch(m, p->bs[b]);
        cudaEventRecord(p->ev_join[b], p->bs[b]);
        cudaStreamWaitEvent(st, p->ev_join[b], 0);
    }
}

}  // namespace

extern "C" const char* rsim_last_error(void) { return g_err.c_str(); }

void rsim::set_last_error(const char* msg) { g_err = msg; }

extern "C" int64_t rsim_plan_scratch_bytes(rsim_plan_t plan) {
    return plan ? (int64_t)plan->dbytes + (plan->rev ? (int64_t)plan->rev->dbytes : 0) +
                      (plan->part ? (int64_t)plan->part->dbytes + (int64_t)plan->part_bytes : 0)
                : 0;
}

extern "C" void rsim_plan_destroy(rsim_plan_t plan) {
    if (!plan) return;
    {
        DeviceGuard g(plan->device);
        for (auto& st : plan->timer.ev)
            for (auto& sl : st)
                for (auto& e : sl)
                    if (e) cudaEventDestroy(e);
        for (int b = 0; b < kNumBuckets; ++b) {
            if (plan->bs[b]) cudaStreamDestroy(plan->bs[b]);
            if (plan->ev_join[b]) cudaEventDestroy(plan->ev_join[b]);
        }
        if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
        plan->gfwd.destroy();
        plan->gbwd.destroy();
        plan->grooms.destroy();
        if (plan->cap) cudaStreamDestroy(plan->cap);
        if (plan->aux) cudaStreamDestroy(plan->aux);
        if (plan->ev_aux) cudaEventDestroy(plan->ev_aux);
        if (plan->ev_plan) cudaEventDestroy(plan->ev_plan);
        if (plan->ev_part) cudaEventDestroy(plan->ev_part);
        if (plan->dmem) cudaFree(plan->dmem);
    }
    if (plan->rev) rsim_plan_destroy(plan->rev);
    if (plan->part) rsim_plan_destroy(plan->part);
    if (plan->part_mem) {
        DeviceGuard g(plan->device);
        cudaFree(plan->part_mem);
    }
    delete plan;
}

namespace {

rsim_status plan_build(const rsim_plan_desc* d, int device, rsim_plan_t* out, rsim_plan_t borrow,
                       int max_sources);

// Builds the partitioned plan over the candidate utterances cand (those whose RIRs reach
// beyond one block of N_max = 2^part_log): its utterance k is utterance cand[k]; virtual
// source (i, q) is source i delayed by q * part_len samples, and its RIR to microphone j is
// taps [q * part_len, (q + 1) * part_len) of h_ij (one zero tap where h_ij is shorter);
// part_len = N_max / 2, ceil(longest RIR of the utterance / part_len) parts.  Every virtual
// signal spans the utterance's output range (N_x, or the full N_x + max N_h - 1), so that
// plan's "same" output is this plan's output, in either output mode.  Its RIRs carry no
// cut-off of their own: the copy of a part holds the taps below the kept length L_ij of this
// plan's cut-off and zeros from there on.  Also builds the copy and sum tables.
rsim_status make_partitioned(rsim_plan_t p, const rsim_plan_desc* d, int device, const std::vector<int32_t>& src0,
                             const std::vector<int32_t>& rir0, const std::vector<int64_t>& xoff,
                             const std::vector<int64_t>& roff, const std::vector<int32_t>& rlen,
                             const std::vector<int64_t>& nyv, const std::vector<int64_t>& yoff, int part_log,
                             const std::vector<int32_t>& cand) {
    const int U = d->num_utts, J = d->num_mics, C = (int)cand.size();
    const bool per_rir = d->gain_mode == 2;       // gains (and their gradients) per RIR
    const int64_t P = (int64_t)1 << (part_log - 1);
    std::vector<int32_t> ns(C), rl;
    std::vector<int64_t> nxs(C);
    // copy tables: x, RIR parts, gains, y (out) and grad_y (in), RIR-gradient parts
    std::vector<int64_t> xs_src, xs_dst, xs_lead, xs_copy, xs_tail, xs_utt;
    std::vector<int64_t> hs_src, hs_dst, hs_copy, hs_tail, hs_utt, hs_limr, hs_limo;
    std::vector<int64_t> as_src, as_dst, as_utt;
    std::vector<int64_t> ys_src, ys_dst, ys_copy, ys_utt;
    // sum tables: dx (over the delayed copies), dalpha (over the parts)
    std::vector<int64_t> dx_out, dx_len, dx_t0{0}, dx_src, dx_tlen, dx_utt;
    std::vector<int64_t> da_out, da_len, da_t0{0}, da_src, da_tlen, da_utt;
    int64_t xv = 0, rv = 0, sv = 0, yv = 0;       // virtual samples, RIR taps, sources, outputs
    for (int k = 0; k < C; ++k) {
        const int u = cand[k];
        const int I = d->num_sources[u];
        const int64_t nx = d->num_samples[u], nv = nyv[u];
        int64_t nh = 1;
        for (int r = rir0[u]; r < rir0[u + 1]; ++r) nh = std::max<int64_t>(nh, rlen[r]);
        const int Pu = (int)((nh + P - 1) / P);
        if ((int64_t)I * Pu > kMaxPartSources)
            return fail(RSIM_E_UNSUPPORTED, "partitioned convolution needs sources x parts <= 64 per utterance");
        ns[k] = I * Pu;
        nxs[k] = nv;
        const int64_t v0 = (int64_t)rl.size();    // this utterance's first virtual RIR
        for (int i = 0; i < I; ++i) {
            const int64_t s = src0[u] + i;
            dx_out.push_back(xoff[s]);
            dx_len.push_back(nx);
            dx_utt.push_back(k);
            for (int q = 0; q < Pu; ++q) {
                const int64_t vq = sv + (int64_t)i * Pu + q;             // virtual source
                const int64_t xq = xv + ((int64_t)i * Pu + q) * nv;      // its samples
                const int64_t lead = std::min<int64_t>((int64_t)q * P, nv);
                const int64_t copy = std::min<int64_t>(nx, nv - lead);
                xs_src.push_back(xoff[s]);
                xs_dst.push_back(xq);
                xs_lead.push_back(lead);
                xs_copy.push_back(copy);
                xs_tail.push_back(nv - lead - copy);
                xs_utt.push_back(k);
                dx_src.push_back(xq + lead);
                dx_tlen.push_back(copy);
                if (!per_rir) {
                    as_src.push_back(s);
                    as_dst.push_back(vq);
                    as_utt.push_back(k);
                    da_src.push_back(vq);
                    da_tlen.push_back(1);
                }
            }
            dx_t0.push_back((int64_t)dx_src.size());
            if (!per_rir) {
                da_out.push_back(s);
                da_len.push_back(1);
                da_utt.push_back(k);
                da_t0.push_back((int64_t)da_src.size());
            }
        }
        // virtual RIRs in (virtual source, microphone) order
        for (int i = 0; i < I; ++i)
            for (int q = 0; q < Pu; ++q)
                for (int j = 0; j < J; ++j) {
                    const int64_t r = rir0[u] + (int64_t)i * J + j;
                    const int64_t valid = std::max<int64_t>(0, std::min<int64_t>(P, rlen[r] - (int64_t)q * P));
                    const int64_t len = std::max<int64_t>(valid, 1);
                    const int64_t vr = (int64_t)rl.size();
                    rl.push_back((int32_t)len);
                    hs_src.push_back(roff[r] + (int64_t)q * P);
                    hs_dst.push_back(rv);
                    hs_copy.push_back(valid);
                    hs_tail.push_back(len - valid);
                    hs_utt.push_back(k);
                    hs_limr.push_back(r);
                    hs_limo.push_back((int64_t)q * P);
                    if (per_rir) {
                        as_src.push_back(r);
                        as_dst.push_back(vr);
                        as_utt.push_back(k);
                    }
                    rv += len;
                }
        if (per_rir) {
            // dalpha_ij sums over the parts: virtual RIR (i, q, j) is the utterance's
            // ((i Pu + q) J + j)-th
            for (int i = 0; i < I; ++i)
                for (int j = 0; j < J; ++j) {
                    da_out.push_back(rir0[u] + (int64_t)i * J + j);
                    da_len.push_back(1);
                    da_utt.push_back(k);
                    for (int q = 0; q < Pu; ++q) {
                        da_src.push_back(v0 + ((int64_t)i * Pu + q) * J + j);
                        da_tlen.push_back(1);
                    }
                    da_t0.push_back((int64_t)da_src.size());
                }
        }
        // the output (J channels of nv samples) and grad_y, one segment each
        ys_src.push_back(yv);
        ys_dst.push_back(yoff[u]);
        ys_copy.push_back((int64_t)J * nv);
        ys_utt.push_back(k);
        yv += (int64_t)J * nv;
        xv += (int64_t)I * Pu * nv;
        sv += (int64_t)I * Pu;
    }
    const int64_t nvr = (int64_t)rl.size();       // virtual RIRs
    rsim_plan_desc pd = *d;
    pd.num_utts = C;
    pd.num_sources = ns.data();
    pd.num_samples = nxs.data();
    pd.rir_len = rl.data();
    pd.eta_db = INFINITY;                         // the parts arrive cut
    pd.gain_mode = per_rir ? 2 : 1;
    pd.output_mode = 0;
    pd.disable_graphs = 1;
    pd.snr_ref_mic = 0;
    pd.rooms = 0;
    pd.long_rirs = 0;
    rsim_status st = plan_build(&pd, device, &p->part, nullptr, kMaxPartSources);
    if (st != RSIM_OK) return fail(st, "partitioned plan: " + g_err);
    if (p->part->part) return fail(RSIM_E_UNSUPPORTED, "partitioned plan: parts beyond one block");
    // one allocation: tables, the deferral flags and indices, then the virtual buffers
    std::vector<int64_t> zeros(std::max<size_t>({xs_src.size(), hs_src.size(), as_src.size(), ys_src.size(),
                                                 (size_t)1}), 0);
    std::vector<int64_t> ones_v(std::max<size_t>(as_src.size(), 1), 1);
    std::vector<int64_t> didx(U, -1);
    for (int k = 0; k < C; ++k) didx[cand[k]] = k;
    struct Arr { const std::vector<int64_t>* v; size_t n; const int64_t** dst; };
    const size_t nS = xs_src.size(), nR = hs_src.size(), nA = as_src.size(), nY = ys_src.size();
    const size_t nO = dx_out.size(), nD = da_out.size();
    const int64_t* defer_idx = nullptr;
    std::vector<Arr> arrs = {
        {&xs_src, nS, &p->seg_x.src}, {&xs_dst, nS, &p->seg_x.dst}, {&xs_lead, nS, &p->seg_x.lead},
        {&xs_copy, nS, &p->seg_x.copy}, {&xs_tail, nS, &p->seg_x.tail}, {&xs_utt, nS, &p->seg_x.utt},
        {&hs_src, nR, &p->seg_h.src}, {&hs_dst, nR, &p->seg_h.dst}, {&zeros, nR, &p->seg_h.lead},
        {&hs_copy, nR, &p->seg_h.copy}, {&hs_tail, nR, &p->seg_h.tail}, {&hs_utt, nR, &p->seg_h.utt},
        {&hs_limr, nR, &p->seg_h.lim_r}, {&hs_limo, nR, &p->seg_h.lim_off},
        {&as_src, nA, &p->seg_a.src}, {&as_dst, nA, &p->seg_a.dst}, {&zeros, nA, &p->seg_a.lead},
        {&ones_v, nA, &p->seg_a.copy}, {&zeros, nA, &p->seg_a.tail}, {&as_utt, nA, &p->seg_a.utt},
        {&hs_dst, nR, &p->seg_dh.src}, {&hs_src, nR, &p->seg_dh.dst}, {&zeros, nR, &p->seg_dh.lead},
        {&hs_copy, nR, &p->seg_dh.copy}, {&zeros, nR, &p->seg_dh.tail}, {&hs_utt, nR, &p->seg_dh.utt},
        {&hs_limr, nR, &p->seg_dh.lim_r}, {&hs_limo, nR, &p->seg_dh.lim_off},
        {&ys_src, nY, &p->seg_y.src}, {&ys_dst, nY, &p->seg_y.dst}, {&zeros, nY, &p->seg_y.lead},
        {&ys_copy, nY, &p->seg_y.copy}, {&zeros, nY, &p->seg_y.tail}, {&ys_utt, nY, &p->seg_y.utt},
        {&ys_dst, nY, &p->seg_gy.src}, {&ys_src, nY, &p->seg_gy.dst}, {&zeros, nY, &p->seg_gy.lead},
        {&ys_copy, nY, &p->seg_gy.copy}, {&zeros, nY, &p->seg_gy.tail}, {&ys_utt, nY, &p->seg_gy.utt},
        {&dx_out, nO, &p->sum_dx.out}, {&dx_len, nO, &p->sum_dx.len}, {&dx_t0, nO + 1, &p->sum_dx.t0},
        {&dx_src, dx_src.size(), &p->sum_dx.src}, {&dx_tlen, dx_tlen.size(), &p->sum_dx.tlen},
        {&dx_utt, nO, &p->sum_dx.utt},
        {&da_out, nD, &p->sum_da.out}, {&da_len, nD, &p->sum_da.len}, {&da_t0, nD + 1, &p->sum_da.t0},
        {&da_src, da_src.size(), &p->sum_da.src}, {&da_tlen, da_tlen.size(), &p->sum_da.tlen},
        {&da_utt, nD, &p->sum_da.utt},
        {&didx, (size_t)U, &defer_idx},
    };
    size_t total = 0;
    for (auto& a : arrs) total = align_up(total, 256) + sizeof(int64_t) * std::max<size_t>(a.n, 1);
    const size_t d_off = align_up(total, 256);
    total = d_off + std::max(C, 1);
    const size_t f_off = align_up(total, 256);
    const int64_t ng = per_rir ? nvr : sv;            // gains: per virtual RIR or virtual source
    const int64_t fl[7] = {xv, rv, ng, yv, xv, rv, ng};    // x, RIR taps, gains, y, dx, dh, dalpha
    total = f_off;
    for (int k = 0; k < 7; ++k) total = align_up(total, 256) + sizeof(float) * std::max<int64_t>(fl[k], 1);
    DeviceGuard guard(device);
    cudaError_t e = cudaMalloc(&p->part_mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RSIM_E_NOMEM, "cudaMalloc of " + std::to_string(total) + " bytes (partitioned) failed");
    }
    p->part_bytes = total;
    size_t off = 0;
    for (auto& a : arrs) {
        off = align_up(off, 256);
        int64_t* dst = (int64_t*)((char*)p->part_mem + off);
        if (a.n) {
            e = cudaMemcpy(dst, a.v->data(), sizeof(int64_t) * a.n, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (partitioned tables)");
        }
        *a.dst = dst;
        off += sizeof(int64_t) * std::max<size_t>(a.n, 1);
    }
    p->defer = (uint8_t*)((char*)p->part_mem + d_off);
    e = cudaMemset(p->defer, 0, std::max(C, 1));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (deferral flags)");
    float** bufs[7] = {&p->part_x, &p->part_rir, &p->part_a, &p->part_y, &p->part_dx, &p->part_dh, &p->part_da};
    off = f_off;
    for (int k = 0; k < 7; ++k) {
        off = align_up(off, 256);
        *bufs[k] = (float*)((char*)p->part_mem + off);
        off += sizeof(float) * std::max<int64_t>(fl[k], 1);
    }
    p->seg_x.n = (int64_t)nS;
    p->seg_h.n = p->seg_dh.n = (int64_t)nR;
    p->seg_a.n = (int64_t)nA;
    p->seg_y.n = p->seg_gy.n = (int64_t)nY;
    p->sum_dx.n = (int64_t)nO;
    p->sum_da.n = (int64_t)nD;
    // destination extents (floats), for the bounds-checked build
    p->seg_x.out_n = xv;
    p->seg_h.out_n = rv;
    p->seg_a.out_n = ng;
    p->seg_y.out_n = yoff[U];
    p->seg_gy.out_n = yv;
    p->seg_dh.out_n = roff.back();
    p->sum_dx.out_n = xoff.back();
    p->sum_da.out_n = per_rir ? (int64_t)roff.size() - 1 : (int64_t)xoff.size() - 1;
    p->part_utt = cand;
    // the outer planner writes the flags the partitioned planner reads; gain mode 2's dalpha
    // reads the RIR parts the forward was given
    p->B.defer_idx = defer_idx;
    p->B.defer = p->defer;
    p->part->B.active = p->defer;
    p->part->fwd_rir = p->part_rir;
    return RSIM_OK;
}

}  // namespace

namespace {
// Builds a plan for description d.  With `borrow` non-NULL the plan takes no new
// device memory, streams or events: its pieces must fit borrow's (same carving
// order, each no larger), which are used at the same offsets (a reshape).
rsim_status plan_build(const rsim_plan_desc* d, int device, rsim_plan_t* out, rsim_plan_t borrow,
                       int max_sources) {
    if (!d || !out) return fail(RSIM_E_INVALID, "rsim_plan: NULL argument");
    *out = nullptr;
    const int U = d->num_utts, J = d->num_mics;
    if (U < 1) return fail(RSIM_E_INVALID, "num_utts must be >= 1");
    if (J < 1 || J > 64) return fail(RSIM_E_INVALID, "num_mics must be in [1, 64]");
    if (!d->num_sources || !d->num_samples || !d->rir_len)
        return fail(RSIM_E_INVALID, "num_sources, num_samples and rir_len are required");
    if (!(d->eta_db >= 0.0)) return fail(RSIM_E_INVALID, "eta_db must be >= 0 or +inf");
    if (d->gain_mode < 0 || d->gain_mode > 3) return fail(RSIM_E_INVALID, "gain_mode must be 0, 1, 2 or 3");
    if (d->gain_mode == 3 && (d->snr_ref_mic < 0 || d->snr_ref_mic >= J))
        return fail(RSIM_E_INVALID, "snr_ref_mic must be in [0, num_mics)");
    int mask = d->fft_sizes_mask;
    const int supported = ((1 << (kMaxLog + 1)) - 1) & ~((1 << kMinLog) - 1);
    if (mask == 0) mask = supported;
    if (mask & ~supported)
        return fail(RSIM_E_UNSUPPORTED, "fft_sizes_mask allows sizes outside 2^11 .. 2^14");
    if (d->output_mode != 0 && d->output_mode != 1) return fail(RSIM_E_INVALID, "output_mode must be 0 or 1");
    if (d->segment_len < 0 || d->bwd_segment_len < 0)
        return fail(RSIM_E_INVALID, "segment_len and bwd_segment_len must be >= 0");
    if (d->long_rirs != 0 && d->long_rirs != 1) return fail(RSIM_E_INVALID, "long_rirs must be 0 or 1");
    if (d->spectrum_cache != 0 && d->spectrum_cache != 1)
        return fail(RSIM_E_INVALID, "spectrum_cache must be 0 or 1");
    // an utterance whose RIRs reach beyond one block of the largest allowed FFT size (hop >=
    // N/4: 3N/4 + 1 taps) gets a partitioned path, without a cut-off or when asked for
    int part_log = kMinLog;
    for (int m = kMinLog; m <= kMaxLog; ++m)
        if ((mask >> m) & 1) part_log = m;
    const int64_t reach = 3 * ((int64_t)1 << part_log) / 4 + 1;
    std::vector<int32_t> cand;
    if (std::isinf(d->eta_db) || d->long_rirs) {
        int64_t r = 0;
        for (int u = 0; u < U; ++u) {
            int64_t nh = 0;
            const int64_t r1 = r + (int64_t)std::max(d->num_sources[u], 0) * J;
            for (; r < r1; ++r) nh = std::max<int64_t>(nh, d->rir_len[r]);
            if (nh > reach) cand.push_back(u);
        }
    }
    const bool partitioned = !cand.empty();
    if (d->rooms != 0 && d->rooms != 1) return fail(RSIM_E_INVALID, "rooms must be 0 or 1");
    if (d->rooms && (partitioned || d->gain_mode == 3))
        return fail(RSIM_E_UNSUPPORTED, "rooms = 1 needs gain_mode 0, 1 or 2 and every RIR within the "
                                        "largest FFT size's reach (no partitioned convolution)");

    std::vector<int32_t> src0(U + 1), rir0(U + 1), seg0(U + 1);
    std::vector<int64_t> yoff(U + 1), nyv(U);
    int64_t S = 0, R = 0, ysz = 0;
    int imax = 1;
    int64_t nx_max = 1;
    int max_log = kMinLog;
    for (int m = kMinLog; m <= kMaxLog; ++m)
        if ((mask >> m) & 1) max_log = m;
    // forward tiles: short segments balance the load across SMs (the backward is
    // cut on the device into one equal-cost chunk per CTA)
    int64_t seg_len = std::max<int64_t>(d->segment_len, (int64_t)1 << max_log);
    int64_t nseg = 0;
    for (int u = 0; u < U; ++u) {
        const int I = d->num_sources[u];
        const int64_t nx = d->num_samples[u];
        if (I < 1 || I > max_sources) return fail(RSIM_E_INVALID, "num_sources[u] must be in [1, 16]");
        if (nx < 1) return fail(RSIM_E_INVALID, "num_samples[u] must be >= 1");
        src0[u] = (int32_t)S;
        rir0[u] = (int32_t)R;
        seg0[u] = (int32_t)nseg;
        yoff[u] = ysz;
        int64_t nh_max = 1;
        for (int64_t r = R; r < R + (int64_t)I * J; ++r) nh_max = std::max<int64_t>(nh_max, d->rir_len[r]);
        nyv[u] = d->output_mode ? nx + nh_max - 1 : nx;
        S += I;
        R += (int64_t)I * J;
        ysz += (int64_t)J * nyv[u];
        nseg += (nx + seg_len - 1) / seg_len;
        imax = std::max(imax, I);
        nx_max = std::max(nx_max, nx);
        if (S > INT32_MAX / 2 || R > INT32_MAX / 2 || nseg > INT32_MAX / 2)
            return fail(RSIM_E_UNSUPPORTED, "batch too large");
    }
    src0[U] = (int32_t)S;
    rir0[U] = (int32_t)R;
    seg0[U] = (int32_t)nseg;
    yoff[U] = ysz;
    std::vector<int32_t> rlen(d->rir_len, d->rir_len + R);
    int nh_max = 1;
    for (int64_t r = 0; r < R; ++r) nh_max = std::max(nh_max, rlen[r]);
    if (d->rooms && nh_max > kCutMaxTaps)
        return fail(RSIM_E_UNSUPPORTED, "rooms = 1 holds each RIR in shared memory: rir_len must be at most 40960");
    std::vector<int64_t> roff(R + 1), xoff(S + 1);
    roff[0] = 0;
    for (int64_t r = 0; r < R; ++r) {
        if (rlen[r] < 1) return fail(RSIM_E_INVALID, "rir_len[r] must be >= 1");
        roff[r + 1] = roff[r] + rlen[r];
    }
    {
        int64_t o = 0;
        for (int u = 0; u < U; ++u)
            for (int i = 0; i < d->num_sources[u]; ++i) {
                xoff[src0[u] + i] = o;
                o += d->num_samples[u];
            }
        xoff[S] = o;
    }
    std::vector<int32_t> src_utt(std::max<int64_t>(S, 1)), rir_utt(std::max<int64_t>(R, 1));
    for (int u = 0; u < U; ++u) {
        for (int s = src0[u]; s < src0[u + 1]; ++s) src_utt[s] = u;
        for (int r = rir0[u]; r < rir0[u + 1]; ++r) rir_utt[r] = u;
    }
    std::vector<int32_t> seg_utt(std::max<int64_t>(nseg, 1));
    int64_t utt_taps_max = 0;                    // RIR taps of the utterance with the most
    for (int u = 0; u < U; ++u) {
        utt_taps_max = std::max<int64_t>(utt_taps_max, roff[rir0[u + 1]] - roff[rir0[u]]);
        for (int g = seg0[u]; g < seg0[u + 1]; ++g) seg_utt[g] = u;
    }
    const int MMAX = 1 << (max_log - 1);
    const int CH = (int)((nx_max + kPowerChunk - 1) / kPowerChunk);

    rsim_plan_t p = new rsim_plan_s();
    p->device = device;
    p->gain_mode = d->gain_mode;
    p->mask = mask;
    p->none = std::isinf(d->eta_db) ? 1 : 0;
    p->factor = p->none ? 0.0 : std::pow(10.0, -d->eta_db / 10.0);

    DeviceGuard guard(device);
    cudaError_t e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }

    // ---- carve one device allocation
    struct Piece { void** dst; size_t bytes; };
    std::vector<Piece> pieces;
    void* p_kept = nullptr;
    void* p_lpre = nullptr;
    void *p_xsoff = nullptr, *p_xspec = nullptr;
    void *p_sord, *p_spre, *p_nstream, *p_ctasp, *p_ctab, *p_ctap, *p_piecedh, *p_sfirst, *p_slast;
    void *p_srcutt, *p_rirutt;
    void *p_nsrc, *p_nx, *p_ny, *p_src0, *p_rir0, *p_seg0, *p_segutt, *p_xoff, *p_yoff, *p_roff, *p_rlen,
        *p_tuning, *p_L, *p_logN, *p_hop, *p_lmax, *p_nblk, *p_pow, *p_err, *p_list,
        *p_count, *p_next, *p_Hc, *p_tails, *p_dhp, *p_dap, *p_melrow, *p_ones, *p_rsrc = nullptr,
        *p_rdst = nullptr, *p_rrir = nullptr, *p_ry = nullptr;
    void* p_tw[2 * kNumBuckets] = {};
    const int64_t cap = std::max<int64_t>(nseg, R);
    // launch shapes (persistent grids) decide the per-CTA backward scratch
    int sms = 0;
    {
        DeviceGuard g0(device);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    }
    if (sms < 1) sms = 1;
    int grid_spec[kNumBuckets] = {}, grid_fwd[kNumBuckets] = {}, grid_bwd[kNumBuckets] = {};
    for (int m = kMinLog; m <= kMaxLog; ++m) {
        if (!((mask >> m) & 1)) continue;
        const int b = m - kMinLog;
        DeviceGuard g0(device);
        grid_spec[b] = (int)std::max<int64_t>(1, std::min<int64_t>(R, (int64_t)sms * occupancy_spectrum(m)));
        grid_fwd[b] = (int)std::max<int64_t>(1, std::min<int64_t>(nseg, (int64_t)sms * occupancy_forward(m)));
        grid_bwd[b] = (int)std::max<int64_t>(1, (int64_t)sms * occupancy_backward(m));
    }
    {
        // test hook, off by default: every persistent launch with one CTA (the work
        // lists and the backward partition then go to a single CTA)
        const char* o = std::getenv("RSIM_TEST_ONE_CTA");
        if (o && o[0] == '1')
            for (int b = 0; b < kNumBuckets; ++b) grid_spec[b] = grid_fwd[b] = grid_bwd[b] = 1;
    }
    // backward partition: at most one piece per stream plus one per CTA boundary; the
    // RIR-gradient partials hold twice the batch's RIR taps (the planner packs the pieces
    // by kept taps and cuts fewer chunks when they would not fit)
    int pmax = 1;
    int64_t ctas = 0;
    for (int b = 0; b < kNumBuckets; ++b) {
        pmax = std::max(pmax, grid_bwd[b]);
        ctas += grid_bwd[b];
    }
    const int64_t npiece = S + ctas;
    const int64_t dhp_total = 2 * roff[R] + 1024;
    (void)utt_taps_max;
    pieces.push_back({&p_nsrc, sizeof(int32_t) * U});
    pieces.push_back({&p_nx, sizeof(int64_t) * U});
    pieces.push_back({&p_ny, sizeof(int64_t) * U});
    pieces.push_back({&p_src0, sizeof(int32_t) * (U + 1)});
    pieces.push_back({&p_rir0, sizeof(int32_t) * (U + 1)});
    pieces.push_back({&p_seg0, sizeof(int32_t) * (U + 1)});
    pieces.push_back({&p_segutt, sizeof(int32_t) * std::max<int64_t>(nseg, 1)});
    pieces.push_back({&p_sord, sizeof(int32_t) * kNumBuckets * std::max<int64_t>(S, 1)});
    pieces.push_back({&p_spre, sizeof(int64_t) * kNumBuckets * (S + 1)});
    pieces.push_back({&p_nstream, sizeof(int32_t) * kNumBuckets});
    pieces.push_back({&p_ctasp, sizeof(int32_t) * kNumBuckets * (pmax + 1)});
    pieces.push_back({&p_ctab, sizeof(int32_t) * kNumBuckets * (pmax + 1)});
    pieces.push_back({&p_ctap, sizeof(int32_t) * kNumBuckets * (pmax + 1)});
    pieces.push_back({&p_piecedh, sizeof(int64_t) * npiece});
    pieces.push_back({&p_lpre, sizeof(int64_t) * (R + 1)});
    pieces.push_back({&p_sfirst, sizeof(int32_t) * std::max<int64_t>(S, 1)});
    pieces.push_back({&p_slast, sizeof(int32_t) * std::max<int64_t>(S, 1)});
    pieces.push_back({&p_xoff, sizeof(int64_t) * (S + 1)});
    pieces.push_back({&p_yoff, sizeof(int64_t) * (U + 1)});
    pieces.push_back({&p_roff, sizeof(int64_t) * (R + 1)});
    pieces.push_back({&p_rlen, sizeof(int32_t) * R});
    pieces.push_back({&p_srcutt, sizeof(int32_t) * std::max<int64_t>(S, 1)});
    pieces.push_back({&p_rirutt, sizeof(int32_t) * std::max<int64_t>(R, 1)});
    pieces.push_back({&p_tuning, sizeof(float) * 32});
    pieces.push_back({&p_L, sizeof(int32_t) * R});
    pieces.push_back({&p_logN, sizeof(int32_t) * U});
    pieces.push_back({&p_hop, sizeof(int32_t) * U});
    pieces.push_back({&p_lmax, sizeof(int32_t) * U});
    pieces.push_back({&p_nblk, sizeof(int32_t) * U});
    pieces.push_back({&p_pow, sizeof(double) * S * CH});
    pieces.push_back({&p_err, sizeof(int32_t) * 4});
    pieces.push_back({&p_list, sizeof(int32_t) * kNumLists * kNumBuckets * cap});
    pieces.push_back({&p_count, sizeof(int32_t) * kNumLists * kNumBuckets});
    pieces.push_back({&p_next, sizeof(int32_t) * kNumLists * kNumBuckets});
    pieces.push_back({&p_Hc, sizeof(float2) * R * MMAX});
    pieces.push_back({&p_tails, sizeof(float) * nseg * J * 2 * MMAX});
    pieces.push_back({&p_dhp, sizeof(float) * std::max<int64_t>(dhp_total, 1)});
    pieces.push_back({&p_dap, sizeof(float) * npiece * kMaxSources});
    pieces.push_back({&p_melrow, sizeof(int64_t) * (U + 1)});
    pieces.push_back({&p_ones, sizeof(float) * std::max<int64_t>(S, 1)});
    if (d->rooms) pieces.push_back({&p_kept, sizeof(float) * std::max<int64_t>(roff[R], 1)});
    // the forward's source spectra for the backward (every size): block b of a source
    // takes 4N bytes and there are at most ceil(4 Nx / N) blocks (hop >= N/4), so at most
    // 16 Nx + 4N bytes per source whatever N the planner picks
    int cache_log = 0;
    for (int m = kMinLog; m <= kMaxLog; ++m)
        if ((mask >> m) & 1) cache_log = m;
    const bool cache = d->spectrum_cache && cache_log > 0;
    std::vector<int64_t> xs_off(S + 1, 0);
    if (cache) {
        for (int u = 0; u < U; ++u)
            for (int s = src0[u]; s < src0[u + 1]; ++s)
                xs_off[s + 1] = xs_off[s] + (int64_t)align_up((size_t)(16 * d->num_samples[u] + (4LL << cache_log)),
                                                              256);
        pieces.push_back({&p_xsoff, sizeof(int64_t) * (S + 1)});
        pieces.push_back({&p_xspec, (size_t)std::max<int64_t>(xs_off[S], 256)});
    }
    // gain_mode 3: each source's RIR to the reference microphone, gathered, and the
    // reverberant sources (laid out like x)
    std::vector<int64_t> rev_src(S), rev_dst(S + 1, 0);
    std::vector<int32_t> rev_len(S);
    if (d->gain_mode == 3) {
        for (int u = 0; u < U; ++u)
            for (int i = 0; i < d->num_sources[u]; ++i) {
                const int64_t s = src0[u] + i, r = rir0[u] + (int64_t)i * J + d->snr_ref_mic;
                rev_src[s] = roff[r];
                rev_len[s] = rlen[r];
                rev_dst[s + 1] = rev_dst[s] + rlen[r];
            }
        pieces.push_back({&p_rsrc, sizeof(int64_t) * std::max<int64_t>(S, 1)});
        pieces.push_back({&p_rdst, sizeof(int64_t) * (S + 1)});
        pieces.push_back({&p_rrir, sizeof(float) * std::max<int64_t>(rev_dst[S], 1)});
        pieces.push_back({&p_ry, sizeof(float) * std::max<int64_t>(xoff[S], 1)});
    }
    std::vector<std::vector<float2>> tws(2 * kNumBuckets);
    for (int m = kMinLog; m <= kMaxLog; ++m) {
        if (!((mask >> m) & 1)) continue;
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * (m - kMinLog) + e;
            tws[k] = twiddle_table_for(m, e ? 16 : 8);
            pieces.push_back({&p_tw[k], sizeof(float2) * tws[k].size()});
        }
    }
    if (borrow) {
        // a reshape: every piece must fit the shape class's
        bool fits = pieces.size() == borrow->piece_cap.size();
        for (size_t k = 0; fits && k < pieces.size(); ++k) fits = pieces[k].bytes <= borrow->piece_cap[k];
        if (!fits) {
            delete p;
            return fail(RSIM_E_UNSUPPORTED, "the batch does not fit the plan's shape class (make a new plan)");
        }
        p->dmem = borrow->dmem;
        p->dbytes = borrow->dbytes;
        p->piece_cap = borrow->piece_cap;
    } else {
        size_t total = 0;
        for (auto& pc : pieces) total = align_up(total, 256) + pc.bytes;
        total = align_up(total, 256);
        e = cudaMalloc(&p->dmem, total);
        if (e != cudaSuccess) {
            delete p;
            cudaGetLastError();
            return fail(RSIM_E_NOMEM, "cudaMalloc of " + std::to_string(total) + " bytes failed");
        }
        p->dbytes = total;
        for (auto& pc : pieces) p->piece_cap.push_back(pc.bytes);
    }
    {
        size_t off = 0;
        for (size_t k = 0; k < pieces.size(); ++k) {
            off = align_up(off, 256);
            *pieces[k].dst = (char*)p->dmem + off;
            off += p->piece_cap[k];
        }
    }
    // ---- uploads
    std::vector<float> tuning(32, 0.f);
    for (int m = 0; m < 32; ++m) tuning[m] = d->fft_cost ? d->fft_cost[m] : (float)((double)m * std::ldexp(1.0, m));
    std::vector<int32_t> nsrc(d->num_sources, d->num_sources + U);
    std::vector<int64_t> nxv(d->num_samples, d->num_samples + U);
    std::vector<float> ones(std::max<int64_t>(S, 1), 1.f);
    struct Up { void* dst; const void* src; size_t bytes; };
    std::vector<Up> ups = {
        {p_nsrc, nsrc.data(), sizeof(int32_t) * U},
        {p_nx, nxv.data(), sizeof(int64_t) * U},
        {p_ny, nyv.data(), sizeof(int64_t) * U},
        {p_src0, src0.data(), sizeof(int32_t) * (U + 1)},
        {p_rir0, rir0.data(), sizeof(int32_t) * (U + 1)},
        {p_seg0, seg0.data(), sizeof(int32_t) * (U + 1)},
        {p_segutt, seg_utt.data(), sizeof(int32_t) * nseg},
        {p_xoff, xoff.data(), sizeof(int64_t) * (S + 1)},
        {p_yoff, yoff.data(), sizeof(int64_t) * (U + 1)},
        {p_roff, roff.data(), sizeof(int64_t) * (R + 1)},
        {p_rlen, rlen.data(), sizeof(int32_t) * R},
        {p_srcutt, src_utt.data(), sizeof(int32_t) * S},
        {p_rirutt, rir_utt.data(), sizeof(int32_t) * R},
        {p_tuning, tuning.data(), sizeof(float) * 32},
        {p_ones, ones.data(), sizeof(float) * ones.size()},
    };
    if (cache) ups.push_back({p_xsoff, xs_off.data(), sizeof(int64_t) * (S + 1)});
    if (d->gain_mode == 3) {
        ups.push_back({p_rsrc, rev_src.data(), sizeof(int64_t) * S});
        ups.push_back({p_rdst, rev_dst.data(), sizeof(int64_t) * (S + 1)});
    }
    for (int k = 0; k < 2 * kNumBuckets; ++k)
        if (p_tw[k]) ups.push_back({p_tw[k], tws[k].data(), sizeof(float2) * tws[k].size()});
    for (auto& up : ups) {
        if (up.bytes == 0) continue;
        e = cudaMemcpy(up.dst, up.src, up.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rsim_plan_destroy(p);
            return cuda_fail(e, "cudaMemcpy (plan upload)");
        }
    }
    e = cudaMemset(p_err, 0, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = cudaMemset(p_count, 0, sizeof(int32_t) * kNumLists * kNumBuckets);
    if (e != cudaSuccess) {
        rsim_plan_destroy(p);
        return cuda_fail(e, "cudaMemset (plan)");
    }

    DevBatch& B = p->B;
    B.U = U; B.J = J; B.S = (int32_t)S; B.R = (int32_t)R; B.IMAX = imax;
    B.NSEG = (int32_t)nseg; B.MMAX = MMAX; B.mask = mask; B.seg_len = seg_len;
    B.PMAX = pmax; B.NPIECE = (int32_t)npiece; B.NDHP = dhp_total;
    B.sord = (int32_t*)p_sord; B.spre = (int64_t*)p_spre; B.nstream = (int32_t*)p_nstream;
    B.cta_sp = (int32_t*)p_ctasp; B.cta_b = (int32_t*)p_ctab; B.cta_p = (int32_t*)p_ctap;
    B.piece_dh = (int64_t*)p_piecedh; B.s_first = (int32_t*)p_sfirst; B.s_last = (int32_t*)p_slast;
    B.lpre = (int64_t*)p_lpre;
    B.xspec = (float4*)p_xspec;
    B.xspec_off = (const int64_t*)p_xsoff;
    B.xspec_bytes = cache ? xs_off[S] : 0;
    // the device planner computes gains from the source powers in modes 0 and 3 (in mode 3
    // the powers are those of the reverberant sources)
    B.gain_mode = d->gain_mode == 3 ? 0 : d->gain_mode;
    B.n_src = (const int32_t*)p_nsrc; B.n_x = (const int64_t*)p_nx; B.n_y = (const int64_t*)p_ny;
    B.src0 = (const int32_t*)p_src0; B.rir0 = (const int32_t*)p_rir0;
    B.seg0 = (const int32_t*)p_seg0; B.seg_utt = (const int32_t*)p_segutt;
    B.xoff = (const int64_t*)p_xoff; B.yoff = (const int64_t*)p_yoff;
    B.roff = (const int64_t*)p_roff; B.rir_len = (const int32_t*)p_rlen;
    B.src_utt = (const int32_t*)p_srcutt; B.rir_utt = (const int32_t*)p_rirutt;
    B.tuning = (const float*)p_tuning;
    B.L = (int32_t*)p_L; B.logN = (int32_t*)p_logN; B.hop = (int32_t*)p_hop;
    B.Lmax = (int32_t*)p_lmax; B.nblk = (int32_t*)p_nblk;
    for (int b = 0; b < kNumBuckets; ++b) B.bgrid[b] = grid_bwd[b];
    B.pow_part = (double*)p_pow; B.CH = CH; B.err = (int32_t*)p_err;
    {
        const char* w = std::getenv("RSIM_TEST_WITHHOLD_BULK_COPY");   // test hook, off by default
        B.test_withhold = (w && w[0] == '1') ? 1 : 0;
    }
    p->Q.list = (int32_t*)p_list; p->Q.count = (int32_t*)p_count; p->Q.next = (int32_t*)p_next;
    p->Q.cap = (int32_t)cap;
    p->Hc = (float2*)p_Hc; p->tails = (float*)p_tails; p->dhp = (float*)p_dhp; p->dap = (float*)p_dap;
    p->mel_row_off = (int64_t*)p_melrow;
    p->ones = (float*)p_ones;
    p->rir_kept = (float*)p_kept;
    p->nh_max = nh_max;
    if (d->rooms) {
        DeviceGuard g0(device);
        p->grid_cut = image_cut_grid(nh_max, (int)R, p->sms);
    }
    p->rev_src_off = (const int64_t*)p_rsrc;
    p->rev_dst_off = (const int64_t*)p_rdst;
    p->rev_rir = (float*)p_rrir;
    p->rev_y = (float*)p_ry;
    p->h_ny = nyv;
    for (int b = 0; b < kNumBuckets; ++b) {
        p->tw[b] = Twiddles{(const float2*)p_tw[2 * b], (const float2*)p_tw[2 * b + 1]};
        p->grid_spec[b] = grid_spec[b];
        p->grid_fwd[b] = grid_fwd[b];
        p->grid_bwd[b] = grid_bwd[b];
    }
    // one CTA per RIR (the scheduler balances their uneven lengths)
    p->grid_trunc = (int)std::max<int64_t>(1, std::min<int64_t>(R, (int64_t)1 << 20));
    // one CTA per chunk (the scheduler balances them; chunks past an utterance's end exit)
    p->grid_pow = (int)std::max<int64_t>(1, std::min<int64_t>(S * CH, (int64_t)1 << 20));
    p->use_graphs = d->disable_graphs == 0;
    p->desc_fixed = *d;
    p->desc_fixed.num_utts = 0;
    p->desc_fixed.num_sources = nullptr;
    p->desc_fixed.num_samples = nullptr;
    p->desc_fixed.rir_len = nullptr;
    p->desc_fixed.fft_cost = nullptr;
    if (borrow) {
        // the streams and events of the shape class (moved over by the reshape)
        p->cap = borrow->cap;
        p->aux = borrow->aux;
        p->ev_aux = borrow->ev_aux;
        p->ev_plan = borrow->ev_plan;
        p->ev_part = borrow->ev_part;
        p->ev_fork = borrow->ev_fork;
        for (int b = 0; b < kNumBuckets; ++b) {
            p->bs[b] = borrow->bs[b];
            p->ev_join[b] = borrow->ev_join[b];
        }
    } else {
        e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_aux, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_plan, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_part, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        for (int m = kMinLog; m <= kMaxLog && e == cudaSuccess; ++m) {
            if (!((mask >> m) & 1)) continue;
            const int b = m - kMinLog;
            e = cudaStreamCreateWithFlags(&p->bs[b], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[b], cudaEventDisableTiming);
        }
    }
    if (e != cudaSuccess) {
        rsim_plan_destroy(p);
        return cuda_fail(e, "stream/event creation");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        rsim_plan_destroy(p);
        return cuda_fail(e, "kernel attribute setup");
    }
    if (partitioned) {
        const rsim_status ps = make_partitioned(p, d, device, src0, rir0, xoff, roff, rlen, nyv, yoff, part_log,
                                                cand);
        if (ps != RSIM_OK) {
            const std::string msg = g_err;
            rsim_plan_destroy(p);
            return fail(ps, msg);
        }
    }
    if (d->gain_mode == 3) {
        // every source its own utterance, one microphone, its RIR to the reference microphone
        std::vector<int32_t> ones_i(S, 1);
        std::vector<int64_t> rev_nx(S);
        for (int u = 0; u < U; ++u)
            for (int i = 0; i < d->num_sources[u]; ++i) rev_nx[src0[u] + i] = d->num_samples[u];
        rsim_plan_desc rd = *d;
        rd.num_utts = (int32_t)S;
        rd.num_mics = 1;
        rd.num_sources = ones_i.data();
        rd.num_samples = rev_nx.data();
        rd.rir_len = rev_len.data();
        rd.gain_mode = 1;
        rd.output_mode = 0;
        rd.disable_graphs = 1;
        rd.snr_ref_mic = 0;
        rd.rooms = 0;
        rd.spectrum_cache = 0;                   // no backward runs on it
        const rsim_status rs = rsim_plan(&rd, device, &p->rev);
        if (rs != RSIM_OK) {
            const std::string msg = "reverberant-SNR plan: " + g_err;
            rsim_plan_destroy(p);
            return fail(rs, msg);
        }
    }
    *out = p;
    return RSIM_OK;
}

}  // namespace

extern "C" rsim_status rsim_plan(const rsim_plan_desc* d, int device, rsim_plan_t* out) {
    g_err.clear();
    return plan_build(d, device, out, nullptr, kMaxSources);
}

extern "C" rsim_status rsim_plan_reshape(rsim_plan_t p, const rsim_plan_desc* d) {
    g_err.clear();
    if (!p || !d) return fail(RSIM_E_INVALID, "rsim_plan_reshape: NULL argument");
    if (p->part || p->rev)
        return fail(RSIM_E_UNSUPPORTED, "plans with partitioned convolution or reverberant-SNR gains "
                                        "cannot be reshaped");
    const rsim_plan_desc& f = p->desc_fixed;
    if (d->num_mics != f.num_mics || d->eta_db != f.eta_db || d->fft_sizes_mask != f.fft_sizes_mask ||
        d->gain_mode != f.gain_mode || d->output_mode != f.output_mode || d->snr_ref_mic != f.snr_ref_mic ||
        d->rooms != f.rooms || d->segment_len != f.segment_len || d->disable_graphs != f.disable_graphs ||
        d->long_rirs != f.long_rirs || d->spectrum_cache != f.spectrum_cache)
        return fail(RSIM_E_INVALID, "rsim_plan_reshape: only the batch shape may change (num_utts, "
                                    "num_sources, num_samples, rir_len, fft_cost)");
    DeviceGuard guard(p->device);
    rsim_plan_t np = nullptr;
    const rsim_status st = plan_build(d, p->device, &np, p, kMaxSources);
    if (st != RSIM_OK) return st;                // p is unchanged
    if (np->part || np->rev) {
        // the new shape needs a sub-plan: keep the old state
        np->dmem = nullptr;
        np->cap = np->aux = nullptr;
        np->ev_aux = np->ev_plan = np->ev_part = np->ev_fork = nullptr;
        for (int b = 0; b < kNumBuckets; ++b) {
            np->bs[b] = nullptr;
            np->ev_join[b] = nullptr;
        }
        rsim_plan_destroy(np);
        return fail(RSIM_E_UNSUPPORTED, "the new shape needs partitioned convolution: make a new plan");
    }
    // no work of the old shape may still read the tables being replaced
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        np->dmem = nullptr;
        np->cap = np->aux = nullptr;
        np->ev_aux = np->ev_plan = np->ev_part = np->ev_fork = nullptr;
        for (int b = 0; b < kNumBuckets; ++b) {
            np->bs[b] = nullptr;
            np->ev_join[b] = nullptr;
        }
        rsim_plan_destroy(np);
        return cuda_fail(e, "cudaDeviceSynchronize (reshape)");
    }
    // the old state (graphs, timer) goes; the memory, streams and events stay with p
    std::swap(*p, *np);
    np->dmem = nullptr;
    np->cap = np->aux = nullptr;
    np->ev_aux = np->ev_plan = np->ev_part = np->ev_fork = nullptr;
    for (int b = 0; b < kNumBuckets; ++b) {
        np->bs[b] = nullptr;
        np->ev_join[b] = nullptr;
    }
    rsim_plan_destroy(np);
    return RSIM_OK;
}

namespace {

// grid: up to 4096 segment rows, and enough blocks per row to cover about 8 blocks per SM
// in all (long segments, such as a deferred utterance's output, then spread over the GPU)
dim3 segs_grid(rsim_plan_t p, int64_t n) {
    const int64_t rows = std::min<int64_t>(n, 4096);
    const int64_t cols = std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)p->sms * 8 + rows - 1) / rows));
    return dim3((unsigned)cols, (unsigned)rows);
}
void copy_segs(rsim_plan_t p, const rsim_plan_s::Segs& g, const float* in, float* out, cudaStream_t st) {
    if (g.n > 0) k_copy_segs<<<segs_grid(p, g.n), 256, 0, st>>>(p->B, g, in, out);
}
void sum_segs(rsim_plan_t p, const rsim_plan_s::Sums& g, const float* in, float* out, cudaStream_t st) {
    if (g.n > 0) k_sum_segs<<<segs_grid(p, g.n), 256, 0, st>>>(p->B, g, in, out);
}

// Room geometry of rsim_filter_mix_rooms: the RIRs are made on the device with
// the cut-off fused (their kept taps land in p->rir_kept)
struct RoomsCall {
    const rsim_image_geom* geom;
    int order;
    float fs, c0;
    float* rir_out;
};

// The forward launch sequence on stream st (eager, or recorded by a capture).
cudaError_t enqueue_forward(rsim_plan_t p, cudaStream_t st, const float* x, const float* rir,
                            const float* snr_db, float* gains, float* y, int32_t* trunc_len,
                            float* energy_kept_frac, const RoomsCall* rooms = nullptr) {
    const DevBatch& B = p->B;
    // the cut-off: the scan of the caller's RIRs, or the RIRs made from room geometry
    // with the cut-off fused, whose kept taps then stand in for the caller's RIRs
    auto cut = [&](cudaStream_t s) {
        if (rooms)
            launch_image_cut(B, rooms->geom, rooms->order, rooms->fs, rooms->c0, p->factor, p->none, p->nh_max,
                             p->rir_kept, rooms->rir_out, energy_kept_frac, p->grid_cut, s);
        else
            launch_truncate(B, rir, p->factor, p->none, energy_kept_frac, p->grid_trunc, s);
    };
    if (rooms) rir = p->rir_kept;
    // per-(i, j) gains fold into the RIR spectra; the kernels then see unit source gains
    const float* rir_gain = p->gain_mode == 2 ? gains : nullptr;
    const float* src_gains = p->gain_mode == 2 ? p->ones : gains;
    bool gains_aside = false;                    // the gains come from the side stream (ev_aux)
    if (p->gain_mode == 3) {
        // reverberant sources at the reference microphone (the auxiliary plan, unit gains),
        // then their powers, turned into gains as for the dry signals
        k_gather_rirs<<<(unsigned)std::min<int64_t>(std::max<int64_t>(B.S, 1), 4096), 256, 0, st>>>(
            B.S, p->rev_src_off, p->rev_dst_off, rir, p->rev_rir);
        cudaError_t e = enqueue_forward(p->rev, st, x, p->rev_rir, nullptr, p->ones, p->rev_y, nullptr, nullptr);
        if (e != cudaSuccess) return e;
        stage_mark(p, 0, false, st);
        launch_truncate(B, rir, p->factor, p->none, energy_kept_frac, p->grid_trunc, st);
        stage_mark(p, 0, true, st);
        stage_mark(p, 1, false, st);
        launch_power(B, p->rev_y, p->grid_pow, st);
        launch_gains(B, snr_db, gains, st);
        stage_mark(p, 1, true, st);
    } else if (p->gain_mode == 0 && !p->timer.on) {
        // source powers (reads x) and the gains run beside the RIR scan (reads rir), the
        // planner and the RIR spectra, which need only the cut-off; each size's forward
        // waits for the gains (ev_aux) after its spectra
        cudaEventRecord(p->ev_fork, st);
        cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
        launch_power(B, x, p->grid_pow, p->aux);
        launch_gains(B, snr_db, gains, p->aux);
        cudaEventRecord(p->ev_aux, p->aux);
        cut(st);
        gains_aside = true;
    } else {
        stage_mark(p, 0, false, st);
        cut(st);
        stage_mark(p, 0, true, st);
        if (p->gain_mode == 0) {
            stage_mark(p, 1, false, st);
            launch_power(B, x, p->grid_pow, st);
            launch_gains(B, snr_db, gains, st);
            stage_mark(p, 1, true, st);
        }
    }
    stage_mark(p, 2, false, st);
    launch_plan(B, p->Q, st);
    if (gains_aside) {
        // the backward partition after the gains on the side stream: it overlaps the
        // spectra and the forward, and the forward's end waits for it
        cudaEventRecord(p->ev_plan, st);
        cudaStreamWaitEvent(p->aux, p->ev_plan, 0);
        launch_partition(B, p->aux);
        cudaEventRecord(p->ev_part, p->aux);
    } else {
        launch_partition(B, st);
    }
    stage_mark(p, 2, true, st);
    if (!p->timer.on) {
        // each FFT size's spectra then its OLA pass on that size's stream: a size's
        // forward waits only for its own spectra
        fan_out(p, st, [&](int m, cudaStream_t s) {
            launch_spectrum(m, B, p->Q, rir, rir_gain, p->Hc, p->tw[m - kMinLog], p->grid_spec[m - kMinLog], s);
            if (gains_aside) cudaStreamWaitEvent(s, p->ev_aux, 0);
            launch_forward(m, B, p->Q, x, src_gains, p->Hc, y, p->tails, p->tw[m - kMinLog],
                           p->grid_fwd[m - kMinLog], s);
        });
    } else {
        stage_mark(p, 3, false, st);
        fan_out(p, st, [&](int m, cudaStream_t s) {
            launch_spectrum(m, B, p->Q, rir, rir_gain, p->Hc, p->tw[m - kMinLog], p->grid_spec[m - kMinLog], s);
        });
        stage_mark(p, 3, true, st);
        stage_mark(p, 4, false, st);
        fan_out(p, st, [&](int m, cudaStream_t s) {
            launch_forward(m, B, p->Q, x, src_gains, p->Hc, y, p->tails, p->tw[m - kMinLog],
                           p->grid_fwd[m - kMinLog], s);
        });
        stage_mark(p, 4, true, st);
    }
    if (gains_aside) cudaStreamWaitEvent(st, p->ev_part, 0);
    stage_mark(p, 5, false, st);
    launch_fixup(B, y, p->tails, st);
    stage_mark(p, 5, true, st);
    if (p->part) {
        // the utterances the planner deferred: their sources delayed by whole parts, their
        // cut RIRs in parts and their gains onto the partitioned plan, its output back
        copy_segs(p, p->seg_x, x, p->part_x, st);
        copy_segs(p, p->seg_h, rir, p->part_rir, st);
        copy_segs(p, p->seg_a, gains, p->part_a, st);
        cudaError_t e = enqueue_forward(p->part, st, p->part_x, p->part_rir, nullptr, p->part_a, p->part_y,
                                        nullptr, nullptr);
        if (e != cudaSuccess) return e;
        copy_segs(p, p->seg_y, p->part_y, y, st);
    }
    if (trunc_len) {
        cudaError_t e = cudaMemcpyAsync(trunc_len, B.L, sizeof(int32_t) * B.R, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// The backward launch sequence on stream st.
cudaError_t enqueue_backward(rsim_plan_t p, cudaStream_t st, const float* grad_y, const float* x,
                             const float* gains, float* grad_x, float* grad_rir, float* grad_gains) {
    const DevBatch& B = p->B;
    const float* rir_gain = p->gain_mode == 2 ? gains : nullptr;
    const float* src_gains = p->gain_mode == 2 ? p->ones : gains;
    cudaError_t e = cudaSuccess;
    stage_mark(p, 6, false, st);
    fan_out(p, st, [&](int m, cudaStream_t s) {
        launch_backward(m, B, p->Q, grad_y, x, src_gains, p->Hc, grad_x, p->dhp, p->dap,
                        p->tw[m - kMinLog], p->grid_bwd[m - kMinLog], s);
    });
    stage_mark(p, 6, true, st);
    stage_mark(p, 7, false, st);
    launch_finalize(B, src_gains, rir_gain, p->fwd_rir, p->dhp, p->dap, grad_rir, grad_gains, st);
    stage_mark(p, 7, true, st);
    if (p->part) {
        // the deferred utterances: grad_y onto the partitioned plan, its gradients folded back
        // over the finalizer's zeros (dx_i sums the delayed copies, dh_ij gathers the parts
        // below the kept length, dalpha sums over the parts)
        copy_segs(p, p->seg_gy, grad_y, p->part_y, st);
        e = enqueue_backward(p->part, st, p->part_y, p->part_x, p->part_a, grad_x ? p->part_dx : nullptr,
                             p->part_dh, p->part_da);
        if (e != cudaSuccess) return e;
        if (grad_x) sum_segs(p, p->sum_dx, p->part_dx, grad_x, st);
        copy_segs(p, p->seg_dh, p->part_dh, grad_rir, st);
        sum_segs(p, p->sum_da, p->part_da, grad_gains, st);
    }
    return cudaGetLastError();
}

// Runs `enqueue` through a CUDA graph captured once per set of buffer
// pointers (key), then replayed on st; eager when graphs are off or stage
// timing is on.
template <typename F>
cudaError_t run_graph(rsim_plan_t p, GraphCache& gc, const void* const (&key)[8], cudaStream_t st, F enqueue) {
    if (!p->use_graphs || p->timer.on) return enqueue(st);
    int slot = -1;
    for (int s = 0; s < kGraphSlots && slot < 0; ++s) {
        bool hit = gc.exec[s] != nullptr;
        for (int k = 0; k < 8 && hit; ++k) hit = gc.key[s][k] == key[k];
        if (hit) slot = s;
    }
    if (slot < 0) {
        slot = 0;                                   // an empty slot, else the least recently used
        for (int s = 0; s < kGraphSlots; ++s) {
            if (!gc.exec[s]) { slot = s; break; }
            if (gc.used[s] < gc.used[slot]) slot = s;
        }
        if (gc.exec[slot]) {
            cudaGraphExecDestroy(gc.exec[slot]);
            gc.exec[slot] = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t le = enqueue(p->cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->cap, &graph);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gc.exec[slot], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gc.exec[slot] = nullptr;
            return e;
        }
        for (int k = 0; k < 8; ++k) gc.key[slot][k] = key[k];
    }
    gc.used[slot] = ++gc.tick;
    return cudaGraphLaunch(gc.exec[slot], st);
}

}  // namespace

extern "C" rsim_status rsim_filter_mix(rsim_plan_t p, void* stream, const float* x, const float* rir,
                                       const float* snr_db, float* gains, float* y, int32_t* trunc_len,
                                       float* energy_kept_frac) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    if (!x || !rir || !gains || !y) return fail(RSIM_E_INVALID, "x, rir, gains and y are required");
    if ((p->gain_mode == 0 || p->gain_mode == 3) && !snr_db)
        return fail(RSIM_E_INVALID, "snr_db is required when gain_mode is 0 or 3");
    DeviceGuard guard(p->device);
    const void* const key[8] = {x, rir, snr_db, gains, y, trunc_len, energy_kept_frac, nullptr};
    cudaError_t e = run_graph(p, p->gfwd, key, (cudaStream_t)stream, [&](cudaStream_t s) {
        return enqueue_forward(p, s, x, rir, snr_db, gains, y, trunc_len, energy_kept_frac);
    });
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    p->fwd_done = true;
    p->fwd_rir = rir;
    return RSIM_OK;
}

extern "C" rsim_status rsim_filter_mix_rooms(rsim_plan_t p, void* stream, const float* x,
                                             const rsim_image_geom* geom, int32_t order, float fs, float c0,
                                             const float* snr_db, float* gains, float* y, int32_t* trunc_len,
                                             float* energy_kept_frac, float* rir_out) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    if (!p->rir_kept) return fail(RSIM_E_STATE, "rsim_filter_mix_rooms needs a plan made with rooms = 1");
    if (!x || !geom || !gains || !y) return fail(RSIM_E_INVALID, "x, geom, gains and y are required");
    if (order < 0 || order > 32 || !(fs > 0.f) || !(c0 > 0.f) || !std::isfinite(fs) || !std::isfinite(c0))
        return fail(RSIM_E_INVALID, "need order in [0, 32] and finite fs, c0 > 0");
    if (p->gain_mode == 0 && !snr_db) return fail(RSIM_E_INVALID, "snr_db is required when gain_mode is 0");
    DeviceGuard guard(p->device);
    // the graphs hold order, fs and c0 by value: other values need new captures
    if (order != p->rooms_order || fs != p->rooms_fs || c0 != p->rooms_c0) {
        p->grooms.destroy();
        p->rooms_order = order;
        p->rooms_fs = fs;
        p->rooms_c0 = c0;
    }
    const RoomsCall rc{geom, order, fs, c0, rir_out};
    const void* const key[8] = {x, geom, snr_db, gains, y, trunc_len, energy_kept_frac, rir_out};
    cudaError_t e = run_graph(p, p->grooms, key, (cudaStream_t)stream, [&](cudaStream_t s) {
        return enqueue_forward(p, s, x, nullptr, snr_db, gains, y, trunc_len, energy_kept_frac, &rc);
    });
    if (e != cudaSuccess) return cuda_fail(e, "forward launch (rooms)");
    p->fwd_done = true;
    p->fwd_rir = p->rir_kept;
    return RSIM_OK;
}

extern "C" rsim_status rsim_filter_mix_backward(rsim_plan_t p, void* stream, const float* grad_y,
                                                const float* x, const float* gains, float* grad_x,
                                                float* grad_rir, float* grad_gains) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    if (!p->fwd_done) return fail(RSIM_E_STATE, "rsim_filter_mix_backward before rsim_filter_mix");
    if (!grad_y || !x || !gains || !grad_rir || !grad_gains)
        return fail(RSIM_E_INVALID, "grad_y, x, gains, grad_rir and grad_gains are required");
    DeviceGuard guard(p->device);
    // the RIR buffer of the last forward is part of the key: the gain gradient of
    // gain mode 2 reads it
    const void* const key[8] = {grad_y, x, gains, grad_x, grad_rir, grad_gains, p->fwd_rir, nullptr};
    cudaError_t e = run_graph(p, p->gbwd, key, (cudaStream_t)stream, [&](cudaStream_t s) {
        return enqueue_backward(p, s, grad_y, x, gains, grad_x, grad_rir, grad_gains);
    });
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    return RSIM_OK;
}

namespace {
// reads and clears the error word of one plan (after the stream was synchronised)
rsim_status check_device_error(rsim_plan_t p) {
    int32_t err = 0;
    cudaError_t e = cudaMemcpy(&err, p->B.err, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (error word)");
    if (err) {
        cudaMemset(p->B.err, 0, sizeof(int32_t));
        if (err & kErrNoFftSize)
            return fail(RSIM_E_UNSUPPORTED,
                        "a truncated RIR is longer than 3N/4+1 for every allowed FFT size N");
        if (err & kErrZeroPower)
            return fail(RSIM_E_INVALID, "a noise source has zero power but an SNR to meet");
        if (err & kErrWaitTimeout)
            return fail(RSIM_E_DEVICE, "a kernel's bounded wait for a bulk copy ran out; results are invalid");
        if (err & kErrBounds)
            return fail(RSIM_E_DEVICE, "bounds-checked build: a kernel store fell outside its buffer (skipped)");
        if (err & kErrBadGeometry)
            return fail(RSIM_E_INVALID, "a room geometry is invalid or puts an image at the microphone "
                                        "(that RIR was taken as all zeros)");
        return fail(RSIM_E_DEVICE, "device error " + std::to_string(err));
    }
    return RSIM_OK;
}
}  // namespace

extern "C" rsim_status rsim_plan_sync_status(rsim_plan_t p, void* stream) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    // the plan's own word, and those of the plans it runs (reverberant gains, partitions)
    rsim_status s = check_device_error(p);
    if (s == RSIM_OK && p->rev) s = check_device_error(p->rev);
    if (s == RSIM_OK && p->part) s = check_device_error(p->part);
    return s;
}

extern "C" rsim_status rsim_plan_query(rsim_plan_t p, void* stream, int32_t* log2_n, int32_t* hop,
                                       int32_t* l_max, int32_t* num_blocks) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    if (!p->fwd_done) return fail(RSIM_E_STATE, "rsim_plan_query before rsim_filter_mix");
    DeviceGuard guard(p->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const size_t n = sizeof(int32_t) * p->B.U;
    if (log2_n && (e = cudaMemcpy(log2_n, p->B.logN, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    if (hop && (e = cudaMemcpy(hop, p->B.hop, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    if (l_max && (e = cudaMemcpy(l_max, p->B.Lmax, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    if (num_blocks && (e = cudaMemcpy(num_blocks, p->B.nblk, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy");
    if (p->part) {
        // deferred utterances report the size, hop and blocks of their partitioned filtering
        // (l_max stays the longest kept RIR)
        const int C = (int)p->part_utt.size();
        std::vector<uint8_t> dfr(C);
        std::vector<int32_t> pl(C), ph(C), pb(C);
        const size_t nc = sizeof(int32_t) * C;
        if ((e = cudaMemcpy(dfr.data(), p->defer, C, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(pl.data(), p->part->B.logN, nc, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(ph.data(), p->part->B.hop, nc, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(pb.data(), p->part->B.nblk, nc, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy");
        for (int k = 0; k < C; ++k) {
            if (!dfr[k]) continue;
            const int u = p->part_utt[k];
            if (log2_n) log2_n[u] = pl[k];
            if (hop) hop[u] = ph[k];
            if (num_blocks) num_blocks[u] = pb[k];
        }
    }
    return RSIM_OK;
}

extern "C" rsim_status rsim_plan_set_timing(rsim_plan_t p, int enable) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    p->timer.on = enable != 0;
    for (int s = 0; s < RSIM_NUM_STAGES; ++s) p->timer.count[s] = 0;
    return RSIM_OK;
}

extern "C" rsim_status rsim_plan_stage_times(rsim_plan_t p, double* ms, int32_t* calls) {
    g_err.clear();
    if (!p) return fail(RSIM_E_INVALID, "NULL plan");
    DeviceGuard guard(p->device);
    for (int s = 0; s < RSIM_NUM_STAGES; ++s) {
        const int n = std::min(p->timer.count[s], kRing);
        double tot = 0.0;
        for (int k = 0; k < n; ++k) {
            cudaEvent_t a = p->timer.ev[s][k][0], b = p->timer.ev[s][k][1];
            cudaError_t e = cudaEventSynchronize(b);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
            float f = 0.f;
            e = cudaEventElapsedTime(&f, a, b);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
            tot += f;
        }
        if (ms) ms[s] = tot;
        if (calls) calls[s] = n;
        p->timer.count[s] = 0;
    }
    return RSIM_OK;
}

// ---- log-Mel front end -------------------------------------------------------
namespace {

rsim_status mel_params(rsim_plan_t p, const rsim_mel_desc* d, MelParams* out) {
    if (!p || !d) return fail(RSIM_E_INVALID, "rsim_plan_log_mel: null plan or description");
    const bool ok = d->channel >= 0 && d->channel < p->B.J && d->hop >= 1 && d->n_mels >= 1 &&
                    d->n_mels <= kMelMaxMels && std::isfinite(d->fs) && d->fs > 0.f && std::isfinite(d->f_lo) &&
                    std::isfinite(d->f_hi) && d->f_lo >= 0.f && d->f_lo < d->f_hi && d->f_hi <= 0.5f * d->fs &&
                    std::isfinite(d->log_floor) && d->log_floor > 0.f && d->stack >= 1 && d->stride >= 1;
    if (!ok)
        return fail(RSIM_E_INVALID, "rsim_plan_log_mel: need 0 <= channel < J, hop >= 1, 1 <= n_mels <= 128, "
                                    "0 <= f_lo < f_hi <= fs / 2, log_floor > 0, stack >= 1, stride >= 1");
    MelParams& m = *out;
    m = MelParams{};
    m.hop = d->hop; m.n_mels = d->n_mels; m.stack = d->stack; m.stride = d->stride;
    m.floor_ = d->log_floor;
    // triangles between n_mels + 2 edges equally spaced on the HTK Mel scale, sampled at the
    // bin frequencies k fs / kMelFft, in FP64; only the nonzero weights are kept
    const auto mel = [](double f) { return 2595.0 * std::log10(1.0 + f / 700.0); };
    const auto hz = [](double v) { return 700.0 * (std::pow(10.0, v / 2595.0) - 1.0); };
    const double m_lo = mel(d->f_lo), m_hi = mel(d->f_hi);
    int nw = 0;
    for (int j = 0; j < d->n_mels; ++j) {
        double e[3];
        for (int q = 0; q < 3; ++q) e[q] = hz(m_lo + (m_hi - m_lo) * (double)(j + q) / (double)(d->n_mels + 1));
        m.off[j] = (int16_t)nw;
        m.first[j] = 0;
        bool started = false;
        for (int k = 0; k <= kMelFft / 2; ++k) {
            const double f = (double)k * (double)d->fs / kMelFft;
            if (!(f > e[0] && f < e[2])) continue;
            const double w = f <= e[1] ? (f - e[0]) / (e[1] - e[0]) : (e[2] - f) / (e[2] - e[1]);
            if (!started) {
                m.first[j] = (int16_t)k;
                started = true;
            }
            if (nw >= kMelMaxWeights) return fail(RSIM_E_INVALID, "rsim_plan_log_mel: filterbank too dense");
            m.w[nw++] = (float)w;
        }
    }
    m.off[d->n_mels] = (int16_t)nw;
    return RSIM_OK;
}

}  // namespace

extern "C" rsim_status rsim_plan_log_mel_rows(rsim_plan_t p, const rsim_mel_desc* d, int64_t* rows_per_utt,
                                              int64_t* total_rows) {
    MelParams mp;
    const rsim_status st = mel_params(p, d, &mp);
    if (st != RSIM_OK) return st;
    int64_t total = 0;
    for (size_t u = 0; u < p->h_ny.size(); ++u) {
        int64_t r, f;
        mel_shape(p->h_ny[u], mp, &r, &f);
        if (rows_per_utt) rows_per_utt[u] = r;
        total += r;
    }
    if (total_rows) *total_rows = total;
    return RSIM_OK;
}

extern "C" rsim_status rsim_plan_log_mel(rsim_plan_t p, void* stream, const float* y, const rsim_mel_desc* d,
                                         float* feats) {
    MelParams mp;
    rsim_status st = mel_params(p, d, &mp);
    if (st != RSIM_OK) return st;
    int64_t frames_max = 0;
    for (int64_t n : p->h_ny) {
        int64_t r, f;
        mel_shape(n, mp, &r, &f);
        frames_max = std::max(frames_max, f);
    }
    // with no rows to write, feats may be null (an empty buffer)
    if (!y || (!feats && frames_max > 0)) return fail(RSIM_E_INVALID, "rsim_plan_log_mel: null y or feats");
    if (frames_max > 0x7fffffff || p->B.U > 65535)
        return fail(RSIM_E_UNSUPPORTED, "rsim_plan_log_mel: more than 65535 utterances or too many frames");
    DeviceGuard guard(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    launch_log_mel(p->B.U, frames_max, y, p->B.yoff, p->B.n_y, d->channel, mp, p->mel_row_off, feats, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "log-Mel launch");
    return RSIM_OK;
}
