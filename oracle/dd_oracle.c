/*
 * dd_oracle.c -- plain, slow, obviously correct CPU oracle for brute-force
 * incoherent dedispersion (Sclocco et al., "Auto-Tuning Dedispersion for
 * Many-Core Accelerators", arXiv:1601.05052).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no source with the CUDA path.
 *
 * Everything is FP64 (or exact int64 for 8-bit input), in the loop order of
 * the paper's Algorithm 1: for every trial DM, for every output sample, sum
 * the channels in ascending channel order.
 *
 * Shift table (Eq. 1, Section II): the delay of channel frequency f relative
 * to the reference frequency f_ref is k = K * DM * (1/f^2 - 1/f_ref^2)
 * seconds, f in MHz, DM in pc/cm^3. The paper prints K ~ 4150; we use the
 * more precise dispersion constant 4.148808e3 MHz^2 s cm^3/pc. The delay in
 * samples is that value divided by the sampling time and rounded to the
 * nearest integer, halves away from zero (C99 llround). Evaluation order:
 * ((K * DM) * (1/(f*f) - 1/(f_ref*f_ref))) / t_samp.
 *
 * OpenMP pragmas only split independent outputs across threads; every output
 * is still summed in ascending channel order by one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_DISPERSION_K 4.148808e3

/* Eq. 1: delay table, row-major [n_dm][n_chan], in samples.
 * Returns 0 on success, -1 on bad arguments (n <= 0, t_samp <= 0, f <= 0),
 * -2 if some shift would be negative (a channel above f_ref with DM > 0). */
int oracle_shift_table(int n_chan, const double *freq_mhz, double f_ref_mhz,
                       double t_samp_s, int n_dm, const double *dm,
                       int64_t *shift_out)
{
    if (n_chan <= 0 || n_dm <= 0 || !(t_samp_s > 0.0) || !(f_ref_mhz > 0.0))
        return -1;
    for (int c = 0; c < n_chan; ++c)
        if (!(freq_mhz[c] > 0.0)) return -1;
    int negative = 0;
    for (int d = 0; d < n_dm; ++d) {
        for (int c = 0; c < n_chan; ++c) {
            double f = freq_mhz[c];
            double inv_f2 = 1.0 / (f * f);
            double inv_ref2 = 1.0 / (f_ref_mhz * f_ref_mhz);
            double delay_s = (ORACLE_DISPERSION_K * dm[d]) * (inv_f2 - inv_ref2);
            double samples = delay_s / t_samp_s;
            long long k = llround(samples);
            if (k < 0) negative = 1;
            shift_out[(int64_t)d * n_chan + c] = (int64_t)k;
        }
    }
    return negative ? -2 : 0;
}

/* Algorithm 1 with per-channel weights, FP64:
 *   out[b][d][t] = sum_c w[c] * in[b][c][t + shift[d][c]]
 * in:  [batch][n_chan][stride] (only the first t_in entries of a row matter)
 * out: [batch][n_dm][n_out]
 * absum (nullable): same shape as out, sum_c |w[c] * in[...]| (the scale the
 * float tolerance is stated against). */
void oracle_forward_f64(int batch, int n_chan, int n_dm, int64_t n_out,
                        int64_t stride, const double *in, const double *w,
                        const int64_t *shift, double *out, double *absum)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < batch; ++b) {
        for (int d = 0; d < n_dm; ++d) {
            for (int64_t t = 0; t < n_out; ++t) {
                double acc = 0.0, aacc = 0.0;
                for (int c = 0; c < n_chan; ++c) {
                    int64_t k = shift[(int64_t)d * n_chan + c];
                    double term = w[c] * in[((int64_t)b * n_chan + c) * stride + t + k];
                    acc += term;
                    aacc += fabs(term);
                }
                int64_t o = ((int64_t)b * n_dm + d) * n_out + t;
                out[o] = acc;
                if (absum) absum[o] = aacc;
            }
        }
    }
}

/* Same sum for 8-bit unsigned input and integer weights, exact in int64. */
void oracle_forward_u8(int batch, int n_chan, int n_dm, int64_t n_out,
                       int64_t stride, const uint8_t *in, const int64_t *wq,
                       const int64_t *shift, int64_t *out)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < batch; ++b) {
        for (int d = 0; d < n_dm; ++d) {
            for (int64_t t = 0; t < n_out; ++t) {
                int64_t acc = 0;
                for (int c = 0; c < n_chan; ++c) {
                    int64_t k = shift[(int64_t)d * n_chan + c];
                    acc += wq[c] * (int64_t)in[((int64_t)b * n_chan + c) * stride + t + k];
                }
                out[((int64_t)b * n_dm + d) * n_out + t] = acc;
            }
        }
    }
}

/* The forward at selected output points only (for full-size problems):
 * out[i] = sum_c w[c] * in[pb[i]][c][pt[i] + shift[pd[i]][c]]. */
void oracle_forward_points_f64(int n_chan, int64_t stride, const double *in_b0,
                               int64_t batch_elems, const double *w,
                               const int64_t *shift, int64_t n_points,
                               const int64_t *pb, const int64_t *pd,
                               const int64_t *pt, double *out, double *absum)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_points; ++i) {
        double acc = 0.0, aacc = 0.0;
        const double *row0 = in_b0 + pb[i] * batch_elems;
        for (int c = 0; c < n_chan; ++c) {
            int64_t k = shift[pd[i] * n_chan + c];
            double term = w[c] * row0[(int64_t)c * stride + pt[i] + k];
            acc += term;
            aacc += fabs(term);
        }
        out[i] = acc;
        if (absum) absum[i] = aacc;
    }
}

/* Adjoint (transpose) of the forward map with respect to the input, written
 * as the literal scatter of the forward's terms:
 *   for every (b, d, t, c): gin[b][c][t + shift[d][c]] += w[c] * g[b][d][t].
 * gin: [batch][n_chan][stride], zeroed here first; entries a forward term
 * never reads stay 0. Serial over (b, d, t) so the sum order is fixed. */
void oracle_adjoint_f64(int batch, int n_chan, int n_dm, int64_t n_out,
                        int64_t stride, const double *g, const double *w,
                        const int64_t *shift, double *gin)
{
    memset(gin, 0, sizeof(double) * (size_t)batch * n_chan * stride);
    for (int b = 0; b < batch; ++b)
        for (int d = 0; d < n_dm; ++d)
            for (int64_t t = 0; t < n_out; ++t) {
                double gv = g[((int64_t)b * n_dm + d) * n_out + t];
                for (int c = 0; c < n_chan; ++c) {
                    int64_t k = shift[(int64_t)d * n_chan + c];
                    gin[((int64_t)b * n_chan + c) * stride + t + k] += w[c] * gv;
                }
            }
}

/* Derivative of <g, out> with respect to the weights:
 *   gw[c] = sum_b sum_d sum_t g[b][d][t] * in[b][c][t + shift[d][c]]. */
void oracle_grad_w_f64(int batch, int n_chan, int n_dm, int64_t n_out,
                       int64_t stride, const double *g, const double *in,
                       const int64_t *shift, double *gw)
{
    #pragma omp parallel for schedule(static)
    for (int c = 0; c < n_chan; ++c) {
        double acc = 0.0;
        for (int b = 0; b < batch; ++b)
            for (int d = 0; d < n_dm; ++d) {
                int64_t k = shift[(int64_t)d * n_chan + c];
                const double *grow = g + ((int64_t)b * n_dm + d) * n_out;
                const double *irow = in + ((int64_t)b * n_chan + c) * stride + k;
                for (int64_t t = 0; t < n_out; ++t) acc += grow[t] * irow[t];
            }
        gw[c] = acc;
    }
}

/* The adjoint at selected input points (for full-size problems): the terms of
 * the forward that read in[b][c][tau] are those (d, t) with t + shift[d][c] =
 * tau and 0 <= t < n_out, so
 *   gin[b][c][tau] = w[c] * sum_d g[b][d][tau - shift[d][c]] over valid t. */
void oracle_adjoint_points_f64(int n_chan, int n_dm, int64_t n_out,
                               const double *g, const double *w,
                               const int64_t *shift, int64_t n_points,
                               const int64_t *pb, const int64_t *pc,
                               const int64_t *ptau, double *out, double *absum)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_points; ++i) {
        double acc = 0.0, aacc = 0.0;
        for (int d = 0; d < n_dm; ++d) {
            int64_t t = ptau[i] - shift[(int64_t)d * n_chan + pc[i]];
            if (t < 0 || t >= n_out) continue;
            double term = w[pc[i]] * g[(pb[i] * n_dm + d) * n_out + t];
            acc += term;
            aacc += fabs(term);
        }
        out[i] = acc;
        if (absum) absum[i] = aacc;
    }
}

/* grad_w for a subset of channels (for full-size problems). */
void oracle_grad_w_channels_f64(int batch, int n_chan, int n_dm, int64_t n_out,
                                int64_t stride, const double *g,
                                const double *in, const int64_t *shift,
                                int64_t n_sel, const int64_t *chans,
                                double *gw, double *absum)
{
    #pragma omp parallel for schedule(dynamic)
    for (int64_t i = 0; i < n_sel; ++i) {
        int64_t c = chans[i];
        double acc = 0.0, aacc = 0.0;
        for (int b = 0; b < batch; ++b)
            for (int d = 0; d < n_dm; ++d) {
                int64_t k = shift[(int64_t)d * n_chan + c];
                const double *grow = g + ((int64_t)b * n_dm + d) * n_out;
                const double *irow = in + ((int64_t)b * n_chan + c) * stride + k;
                for (int64_t t = 0; t < n_out; ++t) {
                    double term = grow[t] * irow[t];
                    acc += term;
                    aacc += fabs(term);
                }
            }
        gw[i] = acc;
        if (absum) absum[i] = aacc;
    }
}

/* 8-bit forward at selected output points, exact in int64. */
void oracle_forward_points_u8(int n_chan, int64_t stride, const uint8_t *in_b0,
                              int64_t batch_elems, const int64_t *wq,
                              const int64_t *shift, int64_t n_points,
                              const int64_t *pb, const int64_t *pd,
                              const int64_t *pt, int64_t *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_points; ++i) {
        int64_t acc = 0;
        const uint8_t *row0 = in_b0 + pb[i] * batch_elems;
        for (int c = 0; c < n_chan; ++c) {
            int64_t k = shift[pd[i] * n_chan + c];
            acc += wq[c] * (int64_t)row0[(int64_t)c * stride + pt[i] + k];
        }
        out[i] = acc;
    }
}
