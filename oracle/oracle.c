/*
 * FP64 CPU oracle for the room simulator's filter-and-mix path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes, in plain loops and in double precision (inputs are the
 * FP32 values of the caller, converted exactly):
 *
 *   Eq. 7  p_th = max_n h_ij[n]^2 * 10^(-eta/10)
 *   Eq. 8  n_c  = min { m : max_{n>m} h^2[n] < p_th }
 *   Eq. 9  hhat_ij[n] = h_ij[n] for 0 <= n <= n_c + 1
 *   Eq. 2  y_j[n] = sum_i alpha_ij (hhat_ij * x_i)[n], evaluated by the
 *          direct time-domain convolution whose cost is Eq. 3, for
 *          n in [0, Nx) (the "same"-length, causal output)
 *   the adjoint of Eq. 2 (gradients with respect to x_i, hhat_ij, alpha_i)
 *   Eq. 6  the paper's overlap-add FFT filtering, one (i, j) at a time, with
 *          its own radix-2 FFT (oracle_mix_ola, used to cross-check and to
 *          give full-batch references quickly)
 *   Eq. 3, 5, 6  the paper's multiplication-count models
 *   Eq. 1  the image-method room impulse response (Sec. 2), h[n] as the sum
 *          of r^g_v / d_v delta[n - ceil(d_v fs / c0)] over the images of
 *          the source in (2K+1)^3 virtual rooms (its readings are listed
 *          above oracle_image_list)
 *   Sec. 3 the log-Mel front end applied after mixing (its readings are
 *          listed above oracle_hz_to_mel).
 *
 * Readings taken where the paper is silent or garbled:
 *   - output length: n in [0, Nx) (Eq. 2 gives no range);
 *   - gains: one alpha_i per source shared by all microphones; alpha_0 = 1
 *     for the target; alpha_i = sqrt(P_0 / P_i * 10^(-SNR_i/10)) with P the
 *     mean square of the dry signal over [0, Nx);
 *   - Eq. 8 uses a strict "<", so a sample whose power equals p_th is kept;
 *     Eq. 9 keeps one sample beyond n_c, so L = min(n_c + 2, Nh);
 *   - an all-zero RIR (max power 0) keeps L = 1;  eta = +inf keeps all taps;
 *   - Eq. 6's block count is a ceiling (the printed floor contradicts the
 *     paper's own 50.8 M figure at N = 2^14).
 *
 * The power comparison h^2 < p_th is made in IEEE double with no fused
 * multiply-add (build with -ffp-contract=off): h^2 of an FP32 value is exact
 * in double, p_th is one rounded product.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_E_INVALID 1

/* ------------------------------------------------------------------------ */
/* Eq. 3, Eq. 5, Eq. 6: multiplication-count models                          */
/* ------------------------------------------------------------------------ */

/* Eq. 3: direct time-domain convolution, I*J*Nx*Nh multiplications. */
double oracle_cost_td(double I, double J, double Nx, double Nh)
{
    return I * J * Nx * Nh;
}

/* Eq. 5: full-length FFT filtering; two FFTs and one IFFT of N/2 log2 N
 * complex multiplications each (x4 real), plus N real multiplications for the
 * half-spectrum product (x2 for complex) per convolution term. */
double oracle_cost_fft(double I, double J, double N)
{
    return I * J * (6.0 * N * log2(N) + 2.0 * N);
}

/* Eq. 6 (ceiling block count): one FFT and one IFFT per block plus the
 * half-spectrum product, and one FFT of the impulse response per (i, j). */
double oracle_cost_ola(double I, double J, double Nx, double Nh, double N)
{
    double hop = N - Nh + 1.0;
    if (hop < 1.0) return INFINITY;
    double blocks = ceil(Nx / hop);
    return I * J * (blocks * (4.0 * N * log2(N) + 2.0 * N) + 2.0 * N * log2(N));
}

/* N = 2^m minimising Eq. 6 over m in [m_lo, m_hi] with N >= Nh. */
int64_t oracle_best_ola_n(double I, double J, double Nx, double Nh, int m_lo, int m_hi)
{
    int64_t best = 0;
    double best_c = INFINITY;
    for (int m = m_lo; m <= m_hi; ++m) {
        double N = ldexp(1.0, m);
        if (N < Nh) continue;
        double c = oracle_cost_ola(I, J, Nx, Nh, N);
        if (c < best_c) { best_c = c; best = (int64_t)N; }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Eq. 7-9: RIR tail cut-off                                                  */
/* ------------------------------------------------------------------------ */

/* Returns the kept length L (>= 1), or -1 for invalid arguments.
 * eta_db = +INFINITY means no cut-off.  peak, e_tot, e_kept may be NULL. */
int64_t oracle_truncate(const double *h, int64_t n_h, double eta_db,
                        double *peak, double *e_tot, double *e_kept)
{
    if (n_h < 1 || !(eta_db >= 0.0)) return -1;   /* also rejects NaN */

    /* Eq. 7: maximum power and threshold */
    double pmax = 0.0;
    for (int64_t n = 0; n < n_h; ++n) {
        double p = h[n] * h[n];
        if (p > pmax) pmax = p;
    }
    double factor = isinf(eta_db) ? 0.0 : pow(10.0, -eta_db / 10.0);
    double p_th = pmax * factor;

    int64_t L;
    if (pmax == 0.0) {
        L = 1;                       /* degenerate all-zero RIR */
    } else {
        /* Eq. 8: smallest m such that every sample after m is below p_th.
         * suffix = max_{n>m} h^2[n], an empty maximum counting as -inf. */
        int64_t n_c = n_h - 1;
        double suffix = -INFINITY;
        for (int64_t m = n_h - 1; m >= 0; --m) {
            if (suffix < p_th) n_c = m;       /* m qualifies; keep the smallest */
            else break;                       /* smaller m cannot qualify */
            double p = h[m] * h[m];
            if (p > suffix) suffix = p;
        }
        /* Eq. 9: keep 0 <= n <= n_c + 1 */
        L = n_c + 2;
        if (L > n_h) L = n_h;
    }

    if (peak) *peak = pmax;
    if (e_tot || e_kept) {
        double et = 0.0, ek = 0.0;
        for (int64_t n = 0; n < n_h; ++n) {
            double p = h[n] * h[n];
            et += p;
            if (n < L) ek += p;
        }
        if (e_tot) *e_tot = et;
        if (e_kept) *e_kept = ek;
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Gains: alpha_i from per-source SNRs (reading of Eq. 2's alpha_ij)          */
/* ------------------------------------------------------------------------ */

/* x: [I][n_x]; snr_db: [I] (entry 0 unused); alpha: [I] out.
 * Returns ORACLE_E_INVALID if a noise source has zero power. */
int oracle_gains(const double *x, int64_t n_x, int32_t I, const double *snr_db,
                 double *alpha)
{
    double p0 = 0.0;
    for (int64_t n = 0; n < n_x; ++n) p0 += x[n] * x[n];
    p0 /= (double)n_x;
    alpha[0] = 1.0;
    for (int32_t i = 1; i < I; ++i) {
        const double *xi = x + (int64_t)i * n_x;
        double pi = 0.0;
        for (int64_t n = 0; n < n_x; ++n) pi += xi[n] * xi[n];
        pi /= (double)n_x;
        if (!(pi > 0.0)) return ORACLE_E_INVALID;
        alpha[i] = sqrt(p0 / pi * pow(10.0, -snr_db[i] / 10.0));
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2 by direct convolution (Eq. 3's form), one utterance                  */
/* ------------------------------------------------------------------------ */

/* x: [I][n_x]; rir: packed RIRs of this utterance in (i, j) order with
 * offsets rir_off[I*J]; L[I*J]: kept lengths; alpha[I];
 * yj: [n_y] out, mic j only: y_j[n] = sum_i alpha_i sum_k hhat_ij[k] x_i[n-k]
 * for n < n_y, with x_i[m] = 0 outside [0, n_x).  n_y = n_x is the "same"
 * output; n_y = n_x + N_h - 1 the full one. */
static void mix_direct_mic(const double *x, int64_t n_x, int64_t n_y, int32_t I, int32_t J, int32_t j,
                           const double *rir, const int64_t *rir_off, const int64_t *L,
                           const double *alpha, double *yj)
{
    for (int64_t n = 0; n < n_y; ++n) yj[n] = 0.0;
    for (int32_t i = 0; i < I; ++i) {
        const double *xi = x + (int64_t)i * n_x;
        const double *h = rir + rir_off[i * J + j];
        int64_t Lij = L[i * J + j];
        for (int64_t n = 0; n < n_y; ++n) {
            double acc = 0.0;
            int64_t kmax = (n < Lij - 1) ? n : Lij - 1;
            int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;
            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];
            yj[n] += alpha[i] * acc;
        }
    }
}

void oracle_mix_direct(const double *x, int64_t n_x, int32_t I, int32_t J,
                       const double *rir, const int64_t *rir_off, const int64_t *L,
                       const double *alpha, double *y)
{
    for (int32_t j = 0; j < J; ++j)
        mix_direct_mic(x, n_x, n_x, I, J, j, rir, rir_off, L, alpha, y + (int64_t)j * n_x);
}

/* Eq. 2 at the output positions n in [n0, n1) only (any n >= 0; positions
 * past n_x belong to the full output).  y: [J][n1 - n0] out.  Used to check
 * sampled outputs of long signals without computing every sample. */
void oracle_mix_window(const double *x, int64_t n_x, int32_t I, int32_t J,
                       const double *rir, const int64_t *rir_off, const int64_t *L,
                       const double *alpha, int64_t n0, int64_t n1, double *y)
{
    const int64_t w = n1 - n0;
    for (int32_t j = 0; j < J; ++j) {
        double *yj = y + (int64_t)j * w;
        for (int64_t n = n0; n < n1; ++n) {
            double sum = 0.0;
            for (int32_t i = 0; i < I; ++i) {
                const double *xi = x + (int64_t)i * n_x;
                const double *h = rir + rir_off[i * J + j];
                int64_t Lij = L[i * J + j];
                int64_t kmax = (n < Lij - 1) ? n : Lij - 1;
                int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;
                double acc = 0.0;
                for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];
                sum += alpha[i] * acc;
            }
            yj[n - n0] = sum;
        }
    }
}

/* Gradient of source i at input positions m in [m0, m1) only:
 * dx_i[m] = alpha_i sum_j sum_{k < L_ij, m+k < n_y} hhat_ij[k] g_j[m+k].
 * g: [J][n_y]; dx: [m1 - m0] out. */
void oracle_dx_window(const double *g, int64_t n_y, int32_t J, int32_t i,
                      const double *rir, const int64_t *rir_off, const int64_t *L,
                      double alpha_i, int64_t m0, int64_t m1, double *dx)
{
    for (int64_t m = m0; m < m1; ++m) {
        double sum = 0.0;
        for (int32_t j = 0; j < J; ++j) {
            const double *gj = g + (int64_t)j * n_y;
            const double *h = rir + rir_off[i * J + j];
            int64_t Lij = L[i * J + j];
            double acc = 0.0;
            for (int64_t k = 0; k < Lij && m + k < n_y; ++k) acc += h[k] * gj[m + k];
            sum += acc;
        }
        dx[m - m0] = alpha_i * sum;
    }
}

/* Gradient of one RIR at taps k in [k0, k1) only:
 * dh_ij[k] = alpha_i sum_{n < n_y} g_j[n] x_i[n - k] for k < L_ij, 0 for k >= L_ij
 * (x_i[m] = 0 outside [0, n_x)).  x_i: [n_x]; g_j: [n_y]; dh: [k1 - k0] out. */
void oracle_dh_window(const double *x_i, int64_t n_x, const double *g_j, int64_t n_y,
                      int64_t L_ij, double alpha_i, int64_t k0, int64_t k1, double *dh)
{
    for (int64_t k = k0; k < k1; ++k) {
        double acc = 0.0;
        if (k < L_ij) {
            int64_t nmax = n_x + k < n_y ? n_x + k : n_y;   /* n - k < n_x */
            for (int64_t n = k; n < nmax; ++n) acc += g_j[n] * x_i[n - k];
        }
        dh[k - k0] = alpha_i * acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of Eq. 2 (one utterance, one source)                               */
/* ------------------------------------------------------------------------ */

/* g: [J][n_y] upstream gradient dLoss/dy (output length n_y as in mix_direct_mic).
 * dx_i[m]    = alpha_i sum_j sum_{k<L_ij} hhat_ij[k] g_j[m+k]      (m+k < n_y)
 * dh_ij[k]   = alpha_i sum_n g_j[n] x_i[n-k]   for k < L_ij, 0 for k >= L_ij
 * dalpha_i   = sum_j sum_n g_j[n] (hhat_ij * x_i)[n]                        */
static void mix_backward_src(const double *x, int64_t n_x, int64_t n_y, int32_t J, int32_t i,
                             const double *rir, const int64_t *rir_off, const int64_t *rir_len,
                             const int64_t *L, const double *alpha, const double *g,
                             double *dx_i, double *dh, double *dalpha_i)
{
    const double *xi = x + (int64_t)i * n_x;
    double da = 0.0;
    for (int64_t m = 0; m < n_x; ++m) dx_i[m] = 0.0;
    for (int32_t j = 0; j < J; ++j) {
        const double *gj = g + (int64_t)j * n_y;
        const double *h = rir + rir_off[i * J + j];
        int64_t Lij = L[i * J + j];
        double *dhij = dh + rir_off[i * J + j];
        /* dx */
        for (int64_t m = 0; m < n_x; ++m) {
            double acc = 0.0;
            for (int64_t k = 0; k < Lij && m + k < n_y; ++k) acc += h[k] * gj[m + k];
            dx_i[m] += alpha[i] * acc;
        }
        /* dh: n runs over the output positions where x_i[n-k] exists */
        for (int64_t k = 0; k < rir_len[i * J + j]; ++k) {
            double acc = 0.0;
            int64_t nend = (n_x + k < n_y) ? n_x + k : n_y;
            if (k < Lij)
                for (int64_t n = k; n < nend; ++n) acc += gj[n] * xi[n - k];
            dhij[k] = alpha[i] * acc;
        }
        /* dalpha: <g_j, hhat_ij * x_i> */
        for (int64_t n = 0; n < n_y; ++n) {
            double acc = 0.0;
            int64_t kmax = (n < Lij - 1) ? n : Lij - 1;
            int64_t kmin = (n - n_x + 1 > 0) ? n - n_x + 1 : 0;
            for (int64_t k = kmin; k <= kmax; ++k) acc += h[k] * xi[n - k];
            da += gj[n] * acc;
        }
    }
    *dalpha_i = da;
}

/* ------------------------------------------------------------------------ */
/* Batch drivers (OpenMP across utterances, mics or sources)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t *src0;     /* [U+1] first source of utterance */
    int64_t *rir0;     /* [U+1] first RIR of utterance */
    int64_t *xoff;     /* [S]   offset of source s in x */
    int64_t *yoff;     /* [U]   offset of utterance in y */
    int64_t *n_y;      /* [U]   output samples per mic */
    int64_t *roff;     /* [R]   offset of RIR r in rir */
} layout_t;

/* output_mode 0: n_y = n_x ("same"); 1: n_y = n_x + max N_h - 1 over the
 * utterance's RIRs (full convolution length of the untruncated RIRs). */
static void layout_build(int32_t U, int32_t J, const int32_t *n_src, const int64_t *n_x,
                         const int32_t *rir_len, int output_mode, layout_t *lo)
{
    lo->src0 = (int64_t *)malloc(sizeof(int64_t) * (U + 1));
    lo->rir0 = (int64_t *)malloc(sizeof(int64_t) * (U + 1));
    lo->yoff = (int64_t *)malloc(sizeof(int64_t) * (U + 1));
    lo->n_y = (int64_t *)malloc(sizeof(int64_t) * (U + 1));
    lo->src0[0] = 0; lo->rir0[0] = 0; lo->yoff[0] = 0;
    for (int32_t u = 0; u < U; ++u) {
        lo->src0[u + 1] = lo->src0[u] + n_src[u];
        lo->rir0[u + 1] = lo->rir0[u] + (int64_t)n_src[u] * J;
        int64_t nh_max = 1;
        for (int64_t r = lo->rir0[u]; r < lo->rir0[u + 1]; ++r)
            if (rir_len[r] > nh_max) nh_max = rir_len[r];
        lo->n_y[u] = output_mode ? n_x[u] + nh_max - 1 : n_x[u];
        lo->yoff[u + 1] = lo->yoff[u] + (int64_t)J * lo->n_y[u];
    }
    int64_t S = lo->src0[U], R = lo->rir0[U];
    lo->xoff = (int64_t *)malloc(sizeof(int64_t) * (S + 1));
    lo->roff = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
    int64_t o = 0;
    for (int32_t u = 0; u < U; ++u)
        for (int64_t s = lo->src0[u]; s < lo->src0[u + 1]; ++s) { lo->xoff[s] = o; o += n_x[u]; }
    lo->xoff[S] = o;
    o = 0;
    for (int64_t r = 0; r < R; ++r) { lo->roff[r] = o; o += rir_len[r]; }
    lo->roff[R] = o;
}

static void layout_free(layout_t *lo)
{
    free(lo->src0); free(lo->rir0); free(lo->xoff); free(lo->yoff); free(lo->roff); free(lo->n_y);
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Truncation of every RIR in a batch (Eq. 7-9).  Returns ORACLE_E_INVALID on
 * bad arguments.  Outputs may be NULL except L. */
int oracle_truncate_batch(int64_t R, const int32_t *rir_len, const double *rir, double eta_db,
                          int64_t *L, double *peak, double *e_tot, double *e_kept, int nthreads)
{
    set_threads(nthreads);
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
    off[0] = 0;
    for (int64_t r = 0; r < R; ++r) off[r + 1] = off[r] + rir_len[r];
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t r = 0; r < R; ++r) {
        double pk, et, ek;
        int64_t l = oracle_truncate(rir + off[r], rir_len[r], eta_db, &pk, &et, &ek);
        if (l < 0) bad = 1;
        L[r] = l;
        if (peak) peak[r] = pk;
        if (e_tot) e_tot[r] = et;
        if (e_kept) e_kept[r] = ek;
    }
    free(off);
    return bad ? ORACLE_E_INVALID : ORACLE_OK;
}

/* Forward over a batch.  gain_mode 0: alpha from snr_db (out in alpha);
 * gain_mode 1: alpha given in alpha.  L: [R] kept lengths (in, from
 * oracle_truncate_batch).  y: [sum J*Ny] out, Ny per output_mode (see
 * layout_build). */
int oracle_forward_batch(int32_t U, int32_t J, const int32_t *n_src, const int64_t *n_x,
                         const int32_t *rir_len, const double *x, const double *rir,
                         const int64_t *L, const double *snr_db, int gain_mode,
                         double *alpha, double *y, int output_mode, int nthreads)
{
    set_threads(nthreads);
    layout_t lo;
    layout_build(U, J, n_src, n_x, rir_len, output_mode, &lo);
    int bad = 0;
    if (gain_mode == 0) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int32_t u = 0; u < U; ++u) {
            int64_t s0 = lo.src0[u];
            if (oracle_gains(x + lo.xoff[s0], n_x[u], n_src[u], snr_db + s0, alpha + s0))
                bad = 1;
        }
    }
    if (!bad) {
        /* per-utterance relative RIR offsets */
        int64_t R = lo.rir0[U];
        int64_t *rel = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
        for (int32_t u = 0; u < U; ++u)
            for (int64_t r = lo.rir0[u]; r < lo.rir0[u + 1]; ++r)
                rel[r] = lo.roff[r] - lo.roff[lo.rir0[u]];
        int64_t UJ = (int64_t)U * J;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t uj = 0; uj < UJ; ++uj) {
            int32_t u = (int32_t)(uj / J), j = (int32_t)(uj % J);
            int64_t s0 = lo.src0[u], r0 = lo.rir0[u];
            mix_direct_mic(x + lo.xoff[s0], n_x[u], lo.n_y[u], n_src[u], J, j,
                           rir + lo.roff[r0], rel + r0, L + r0, alpha + s0,
                           y + lo.yoff[u] + (int64_t)j * lo.n_y[u]);
        }
        free(rel);
    }
    layout_free(&lo);
    return bad ? ORACLE_E_INVALID : ORACLE_OK;
}

/* Backward over a batch.  g: [sum J*Ny] (Ny per output_mode); dx: [sum I*Nx];
 * dh: like rir; dalpha: [sum I].  alpha and L as used by the forward. */
int oracle_backward_batch(int32_t U, int32_t J, const int32_t *n_src, const int64_t *n_x,
                          const int32_t *rir_len, const double *x, const double *rir,
                          const int64_t *L, const double *alpha, const double *g,
                          double *dx, double *dh, double *dalpha, int output_mode, int nthreads)
{
    set_threads(nthreads);
    layout_t lo;
    layout_build(U, J, n_src, n_x, rir_len, output_mode, &lo);
    int64_t S = lo.src0[U], R = lo.rir0[U];
    int64_t *rel = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
    int64_t *rlen64 = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
    int32_t *utt_of = (int32_t *)malloc(sizeof(int32_t) * (S + 1));
    for (int32_t u = 0; u < U; ++u) {
        for (int64_t r = lo.rir0[u]; r < lo.rir0[u + 1]; ++r) {
            rel[r] = lo.roff[r] - lo.roff[lo.rir0[u]];
            rlen64[r] = rir_len[r];
        }
        for (int64_t s = lo.src0[u]; s < lo.src0[u + 1]; ++s) utt_of[s] = u;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < S; ++s) {
        int32_t u = utt_of[s];
        int32_t i = (int32_t)(s - lo.src0[u]);
        int64_t s0 = lo.src0[u], r0 = lo.rir0[u];
        mix_backward_src(x + lo.xoff[s0], n_x[u], lo.n_y[u], J, i,
                         rir + lo.roff[r0], rel + r0, rlen64 + r0, L + r0, alpha + s0,
                         g + lo.yoff[u], dx + lo.xoff[s], dh + lo.roff[r0], dalpha + s);
    }
    free(rel); free(rlen64); free(utt_of);
    layout_free(&lo);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 4 / Eq. 6: the paper's OLA FFT filtering in FP64, own radix-2 FFT      */
/* ------------------------------------------------------------------------ */

/* In-place iterative radix-2 complex DFT of length n (a power of two);
 * sign = -1 forward, +1 inverse (unnormalised).  re, im: [n]. */
static void fft_radix2(double *re, double *im, int64_t n, int sign)
{
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t k = 0; k < half; ++k) {
            double ang = sign * 2.0 * M_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int64_t s = 0; s < n; s += len) {
                int64_t a = s + k, b = s + k + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] += tr; im[a] += ti;
            }
        }
    }
}

/* Exposed for tests: forward DFT of a real signal x[n] zero-padded to n_fft;
 * out_re/out_im: [n_fft]. */
void oracle_dft_real(const double *x, int64_t n, int64_t n_fft, double *out_re, double *out_im)
{
    for (int64_t k = 0; k < n_fft; ++k) { out_re[k] = k < n ? x[k] : 0.0; out_im[k] = 0.0; }
    fft_radix2(out_re, out_im, n_fft, -1);
}

/* One utterance.  Each (i, j) is filtered on its own, as in the paper: its
 * FFT size N is fft_n if > 0 (must be a power of two >= L_ij), otherwise the
 * 2^m in [2^6, 2^20] minimising Eq. 6 for this (Nx, L_ij); hop = N - L_ij + 1;
 * ceil(Nx / hop) blocks; the RIR spectrum is computed once per (i, j).
 * Output y: [J][n_x], "same" length.  Returns ORACLE_E_INVALID on bad N. */
int oracle_mix_ola(const double *x, int64_t n_x, int32_t I, int32_t J,
                   const double *rir, const int64_t *rir_off, const int64_t *L,
                   const double *alpha, int64_t fft_n, double *y)
{
    for (int64_t n = 0; n < (int64_t)J * n_x; ++n) y[n] = 0.0;
    for (int32_t i = 0; i < I; ++i) {
        const double *xi = x + (int64_t)i * n_x;
        for (int32_t j = 0; j < J; ++j) {
            const double *h = rir + rir_off[i * J + j];
            int64_t Lh = L[i * J + j];
            int64_t N = fft_n > 0 ? fft_n
                                  : oracle_best_ola_n(1.0, 1.0, (double)n_x, (double)Lh, 6, 20);
            if (N < Lh || (N & (N - 1)) != 0) return ORACLE_E_INVALID;
            int64_t hop = N - Lh + 1;
            double *Hr = (double *)malloc(sizeof(double) * N);
            double *Hi = (double *)malloc(sizeof(double) * N);
            double *Br = (double *)malloc(sizeof(double) * N);
            double *Bi = (double *)malloc(sizeof(double) * N);
            oracle_dft_real(h, Lh, N, Hr, Hi);                 /* once per RIR */
            double *yj = y + (int64_t)j * n_x;
            int64_t nblk = (n_x + hop - 1) / hop;
            for (int64_t b = 0; b < nblk; ++b) {
                int64_t s = b * hop;
                int64_t len = (s + hop <= n_x) ? hop : n_x - s;
                oracle_dft_real(xi + s, len, N, Br, Bi);
                for (int64_t k = 0; k < N; ++k) {             /* spectrum product */
                    double r = Br[k] * Hr[k] - Bi[k] * Hi[k];
                    double m = Br[k] * Hi[k] + Bi[k] * Hr[k];
                    Br[k] = r; Bi[k] = m;
                }
                fft_radix2(Br, Bi, N, +1);
                for (int64_t n = 0; n < N && s + n < n_x; ++n)  /* overlap-add */
                    yj[s + n] += alpha[i] * Br[n] / (double)N;
            }
            free(Hr); free(Hi); free(Br); free(Bi);
        }
    }
    return ORACLE_OK;
}

/* Batch form of oracle_mix_ola (OpenMP across utterances). */
int oracle_forward_ola_batch(int32_t U, int32_t J, const int32_t *n_src, const int64_t *n_x,
                             const int32_t *rir_len, const double *x, const double *rir,
                             const int64_t *L, const double *alpha, int64_t fft_n,
                             double *y, int nthreads)
{
    set_threads(nthreads);
    layout_t lo;
    layout_build(U, J, n_src, n_x, rir_len, 0, &lo);
    int64_t R = lo.rir0[U];
    int64_t *rel = (int64_t *)malloc(sizeof(int64_t) * (R + 1));
    for (int32_t u = 0; u < U; ++u)
        for (int64_t r = lo.rir0[u]; r < lo.rir0[u + 1]; ++r)
            rel[r] = lo.roff[r] - lo.roff[lo.rir0[u]];
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t u = 0; u < U; ++u) {
        int64_t s0 = lo.src0[u], r0 = lo.rir0[u];
        if (oracle_mix_ola(x + lo.xoff[s0], n_x[u], n_src[u], J, rir + lo.roff[r0], rel + r0,
                           L + r0, alpha + s0, fft_n, y + lo.yoff[u]))
            bad = 1;
    }
    free(rel);
    layout_free(&lo);
    return bad ? ORACLE_E_INVALID : ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: image-method room impulse response                                 */
/* ------------------------------------------------------------------------ */
/*
 * Readings of Sec. 2 and Eq. 1:
 *  - the room is the box [0, Lx] x [0, Ly] x [0, Lz] (metres); mirroring it
 *    across its walls, again and again, tiles space with virtual rooms indexed
 *    (a, b, c), each index in [-K, K] (K = 8 gives the paper's 17^3 = 4913);
 *    every virtual room holds one image of the source;
 *  - along one axis, virtual room a spans [a L, (a + 1) L]; each mirroring
 *    flips the source coordinate, so the image sits at a L + s for even a and
 *    at (a + 1) L - s for odd a, and it took |a| reflections to get there;
 *    g_v = |a| + |b| + |c|;
 *  - all walls share one reflection coefficient r, 0 <= r < 1 (r = 0 keeps the
 *    direct path alone, r^0 = 1);
 *  - the delay is ceil(t_v) with t_v = d_v fs / c0 the travel time in
 *    samples, evaluated in FP64 from the FP32 geometry (image coordinate,
 *    offset to the microphone, distance, travel time), as is the amplitude
 *    r^g_v / d_v.  Eq. 1 fixes no precision; where t_v lies within a few
 *    FP32 rounding errors of an integer, an FP32 evaluation of the same real
 *    number may land the image one sample later or earlier, and both taps
 *    are readings of Eq. 1 (the travel time is returned so a caller can tell
 *    those images apart);
 *  - an image whose delay is n_h or later lies outside the RIR and is dropped;
 *  - the source and the microphone lie strictly inside the room, and no image
 *    may sit at distance zero from the microphone (d_v > 0, Eq. 1).
 */

static int image_geom_valid(const float *room, const float *src, const float *mic, float refl)
{
    for (int k = 0; k < 3; ++k) {
        if (!(room[k] > 0.0f) || !isfinite(room[k])) return 0;
        if (!(src[k] > 0.0f && src[k] < room[k])) return 0;
        if (!(mic[k] > 0.0f && mic[k] < room[k])) return 0;
    }
    return refl >= 0.0f && refl < 1.0f;
}

/* offset from the microphone to the image coordinate of virtual room a */
static double image_offset_f64(int a, double len, double s, double m)
{
    double p = (a % 2 == 0) ? (double)a * len + s : (double)(a + 1) * len - s;
    return p - m;
}

typedef struct {
    double pos[3];  /* image position (FP64) */
    int32_t g;      /* reflections */
    double travel;  /* d fs / c0 in samples (FP64) */
    int64_t delay;  /* ceil(travel) */
    double amp;     /* r^g / d, FP64 */
    int ok;         /* 0: the image is at distance zero */
} image_t;

static image_t image_eval(const float *room, const float *src, const float *mic, float refl,
                          int a, int b, int c, float fs, float c0)
{
    image_t im;
    const int idx[3] = {a, b, c};
    double e2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double ed = image_offset_f64(idx[k], room[k], src[k], mic[k]);
        im.pos[k] = ed + (double)mic[k];
        e2 += ed * ed;
    }
    im.ok = e2 > 0.0;
    const double d = sqrt(e2);
    im.travel = d * (double)fs / (double)c0;
    /* a travel time beyond any RIR length */
    im.delay = im.travel < 1e18 ? (int64_t)ceil(im.travel) : INT64_MAX;
    im.g = abs(a) + abs(b) + abs(c);
    im.amp = im.ok ? pow((double)refl, (double)im.g) / d : 0.0;
    return im;
}

/* Every image of one (source, microphone) pair, rooms in (a, b, c) order with
 * c fastest.  Arrays hold (2K+1)^3 entries.  Returns the count, or -1 if the
 * arguments are invalid. */
int64_t oracle_image_list(const float *room, const float *src, const float *mic, float refl,
                          int32_t order, float fs, float c0, double *pos, int32_t *g,
                          int64_t *delay, double *amp, double *travel)
{
    if (order < 0 || !(fs > 0.0f) || !(c0 > 0.0f) || !isfinite(fs) || !isfinite(c0)) return -1;
    if (!image_geom_valid(room, src, mic, refl)) return -1;
    int64_t v = 0;
    for (int a = -order; a <= order; ++a)
        for (int b = -order; b <= order; ++b)
            for (int c = -order; c <= order; ++c, ++v) {
                image_t im = image_eval(room, src, mic, refl, a, b, c, fs, c0);
                if (!im.ok) return -1;
                for (int k = 0; k < 3; ++k) pos[3 * v + k] = im.pos[k];
                g[v] = im.g;
                delay[v] = im.delay;
                amp[v] = im.amp;
                travel[v] = im.travel;
            }
    return v;
}

/* Eq. 1: h[n] = sum_v r^g_v / d_v delta[n - ceil(d_v fs / c0)] for n < n_h.
 * h is zeroed first.  Returns the number of images that landed in [0, n_h),
 * or -1 (h left zero) if the arguments are invalid. */
int64_t oracle_image_rir(const float *room, const float *src, const float *mic, float refl,
                         int32_t order, float fs, float c0, int64_t n_h, double *h)
{
    if (n_h < 0 || n_h > ((int64_t)1 << 24)) return -1;
    for (int64_t n = 0; n < n_h; ++n) h[n] = 0.0;
    if (order < 0 || !(fs > 0.0f) || !(c0 > 0.0f) || !isfinite(fs) || !isfinite(c0)) return -1;
    if (!image_geom_valid(room, src, mic, refl)) return -1;
    int64_t landed = 0;
    for (int a = -order; a <= order; ++a)
        for (int b = -order; b <= order; ++b)
            for (int c = -order; c <= order; ++c) {
                image_t im = image_eval(room, src, mic, refl, a, b, c, fs, c0);
                if (!im.ok) {
                    for (int64_t n = 0; n < n_h; ++n) h[n] = 0.0;
                    return -1;
                }
                if (im.delay < n_h) {
                    h[im.delay] += im.amp;
                    ++landed;
                }
            }
    return landed;
}

/* Batch form: RIR r has geometry geom[10 r .. 10 r + 9] = room (3), source (3),
 * microphone (3), r; its taps are h[off[r] .. off[r + 1]).  valid[r] = 1 if its
 * arguments were valid (an invalid RIR is left zero).  OpenMP across RIRs. */
void oracle_image_rirs(int64_t R, const float *geom, const int64_t *off, int32_t order, float fs,
                       float c0, double *h, int32_t *valid, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < R; ++r) {
        const float *gr = geom + 10 * r;
        valid[r] = oracle_image_rir(gr, gr + 3, gr + 6, gr[9], order, fs, c0, off[r + 1] - off[r],
                                    h + off[r]) >= 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: the log-Mel front end after mixing                                */
/* ------------------------------------------------------------------------ */
/*
 * The paper's features: a single channel, 128 log-Mel energies from a 32 ms
 * window every 10 ms, a Mel filterbank from 125 Hz to 7500 Hz, four frames
 * stacked and the stacked frames kept every third.  Readings where it is
 * silent:
 *  - frame t covers samples [t hop, t hop + n_fft) of the channel, with no
 *    padding: T = (n - n_fft) / hop + 1 frames (none if n < n_fft);
 *  - periodic Hann window w[n] = 1/2 - 1/2 cos(2 pi n / n_fft);
 *  - power spectrum |X[k]|^2 of the windowed frame, k = 0 .. n_fft/2;
 *  - HTK Mel scale m(f) = 2595 log10(1 + f/700); n_mels + 2 points equally
 *    spaced in m from m(f_lo) to m(f_hi); filter j is the triangle rising from
 *    point j to point j+1 and falling to point j+2 (peak 1, no area
 *    normalisation), sampled at the bin frequencies k fs / n_fft;
 *  - feature = ln(E + floor) of each filter's energy E;
 *  - stacked row r holds frames stride r .. stride r + stack - 1 side by side
 *    (frame-major), for every r whose frames all exist.
 */

double oracle_hz_to_mel(double f) { return 2595.0 * log10(1.0 + f / 700.0); }

double oracle_mel_to_hz(double m) { return 700.0 * (pow(10.0, m / 2595.0) - 1.0); }

/* weights W[j * (n_fft/2 + 1) + k] of the triangular Mel filters */
void oracle_mel_filters(int32_t n_fft, double fs, int32_t n_mels, double f_lo, double f_hi, double *W)
{
    const int32_t nb = n_fft / 2 + 1;
    const double m_lo = oracle_hz_to_mel(f_lo), m_hi = oracle_hz_to_mel(f_hi);
    for (int32_t j = 0; j < n_mels; ++j) {
        double edge[3];
        for (int e = 0; e < 3; ++e)
            edge[e] = oracle_mel_to_hz(m_lo + (m_hi - m_lo) * (double)(j + e) / (double)(n_mels + 1));
        for (int32_t k = 0; k < nb; ++k) {
            double f = (double)k * fs / (double)n_fft, w = 0.0;
            if (f > edge[0] && f < edge[2])
                w = (f <= edge[1]) ? (f - edge[0]) / (edge[1] - edge[0]) : (edge[2] - f) / (edge[2] - edge[1]);
            W[(int64_t)j * nb + k] = w;
        }
    }
}

/* power spectrum |X[k]|^2, k = 0 .. n_fft/2, of the Hann-windowed frame */
void oracle_frame_power(const double *x, int32_t n_fft, double *P)
{
    double *re = (double *)malloc(sizeof(double) * n_fft), *im = (double *)malloc(sizeof(double) * n_fft);
    for (int32_t n = 0; n < n_fft; ++n) {
        re[n] = x[n] * (0.5 - 0.5 * cos(2.0 * M_PI * (double)n / (double)n_fft));
        im[n] = 0.0;
    }
    fft_radix2(re, im, n_fft, -1);
    for (int32_t k = 0; k <= n_fft / 2; ++k) P[k] = re[k] * re[k] + im[k] * im[k];
    free(re);
    free(im);
}

/* rows of stacked features from n samples */
int64_t oracle_log_mel_rows(int64_t n, int32_t n_fft, int32_t hop, int32_t stack, int32_t stride)
{
    int64_t T = n >= n_fft ? (n - n_fft) / hop + 1 : 0;
    return T >= stack ? (T - stack) / stride + 1 : 0;
}

/* Log-Mel features of one channel of n samples: out[r * stack * n_mels + s * n_mels + j].
 * Returns the number of rows. */
int64_t oracle_log_mel(const double *y, int64_t n, int32_t n_fft, int32_t hop, double fs, int32_t n_mels,
                       double f_lo, double f_hi, double floor_, int32_t stack, int32_t stride, double *out)
{
    const int32_t nb = n_fft / 2 + 1;
    const int64_t rows = oracle_log_mel_rows(n, n_fft, hop, stack, stride);
    if (rows == 0) return 0;
    const int64_t frames = (rows - 1) * stride + stack;
    double *W = (double *)malloc(sizeof(double) * n_mels * nb);
    double *P = (double *)malloc(sizeof(double) * nb);
    double *F = (double *)malloc(sizeof(double) * frames * n_mels);
    oracle_mel_filters(n_fft, fs, n_mels, f_lo, f_hi, W);
    for (int64_t t = 0; t < frames; ++t) {
        oracle_frame_power(y + t * hop, n_fft, P);
        for (int32_t j = 0; j < n_mels; ++j) {
            double e = 0.0;
            for (int32_t k = 0; k < nb; ++k) e += W[(int64_t)j * nb + k] * P[k];
            F[t * n_mels + j] = log(e + floor_);
        }
    }
    for (int64_t r = 0; r < rows; ++r)
        for (int32_t s = 0; s < stack; ++s)
            for (int32_t j = 0; j < n_mels; ++j)
                out[(r * stack + s) * n_mels + j] = F[(r * stride + s) * n_mels + j];
    free(W);
    free(P);
    free(F);
    return rows;
}

/* Batch form over utterances: channel `ch` of y laid out [sum_u J * n_y[u]]
 * (utterance, microphone, sample); rows of utterance u start at row_off[u]
 * (the prefix sum of oracle_log_mel_rows).  OpenMP across utterances. */
void oracle_log_mel_batch(int32_t U, int32_t J, const int64_t *n_y, const double *y, int32_t ch, int32_t n_fft,
                          int32_t hop, double fs, int32_t n_mels, double f_lo, double f_hi, double floor_,
                          int32_t stack, int32_t stride, const int64_t *row_off, double *out, int nthreads)
{
    set_threads(nthreads);
    int64_t *yoff = (int64_t *)malloc(sizeof(int64_t) * (U + 1));
    yoff[0] = 0;
    for (int32_t u = 0; u < U; ++u) yoff[u + 1] = yoff[u] + (int64_t)J * n_y[u];
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t u = 0; u < U; ++u)
        oracle_log_mel(y + yoff[u] + (int64_t)ch * n_y[u], n_y[u], n_fft, hop, fs, n_mels, f_lo, f_hi, floor_,
                       stack, stride, out + row_off[u] * (int64_t)stack * n_mels);
    free(yoff);
}
