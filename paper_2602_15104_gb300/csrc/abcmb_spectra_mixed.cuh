// Mixed-precision line-of-sight projection and k-quadrature (the FP32 form
// of App. B.4 transfer functions and eq. c_ell_def; App. B.6 trapezoid rules).
// The ODE sources stay FP64; here everything per (node, l) point runs on the
// FP32 pipe, which on GB300 issues ~64x faster than FP64:
//
//  * x = k (tau_0 - tau), 1/x, sin x, cos x and the starting j_0, j_1, j_2 in
//    FP64 once per node (FP64 argument reduction), then the upward Bessel
//    recurrence j_{l+1} = (2l+1)/x j_l - j_{l-1} in double-float (a value is
//    an unevaluated pair hi + lo of floats; Dekker's and Knuth's error-free
//    product and sum, ~2^-44 relative).  Plain FP32 cannot run it: its
//    rounding is amplified by the growing solution past the turning point,
//    and a float 1/x alone shifts the phase by x 2^-24 (1e-4 at x ~ 2000).
//  * The collapsed temperature kernel (A0 + l A1 + l^2 A2) j_l + B j_{l-1}
//    and the E kernel E j_l (see abcmb_spectra.cuh) in FP32 on the float j_l;
//    per-lane partial sums over 4 nodes, a 32-lane butterfly reduce-scatter
//    over 128 nodes, then a Kahan-compensated FP32 accumulator per
//    (l, T/E) in shared memory across the node groups.  One warp per
//    (cosmology, k), so each accumulator has a single writer.
//  * Below x = 1 j_l comes from its power series, in FP32.
//  * C_l: FP32 products Delta_X Delta_Y w_k P(k) with Kahan-compensated FP32
//    sums over k; the weights w_k P(k) are formed in FP64.
#pragma once

#include <math.h>

#include "abcmb_bg.cuh"

namespace abcmb {

namespace mixed {

constexpr int kNodesPerLane = 4;
constexpr int kLB = 16;     // l per block
constexpr int kSerL = 32;   // series table rows (l)
constexpr float kSeriesX = 1.0f;

// Debye cutoff of abcmb_spectra.cuh (exponent 16, plus 2 ln(1/x) below x = 1)
__device__ __forceinline__ int bessel_cut_f(float x, int lmax)
{
    if (x > (float)lmax + 200.0f) return lmax;
    const float T = 16.0f + 2.0f * fmaxf(0.0f, -logf(x));
    float nu = x + 1.0f + 0.8f * cbrtf(fmaxf(x, 1.0f)) * 9.0f;
    for (int it = 0; it < 8; it++) {
        float r = fmaxf(nu / fmaxf(x, 1e-30f), 1.0f + 1e-6f);
        float al = acoshf(r);
        float f = nu * (al - tanhf(al)) - T;
        nu = fmaxf(nu - f / fmaxf(al, 1e-3f), x + 0.5f);
    }
    int l = (int)ceilf(nu - 0.5f);
    return l < 2 ? 2 : (l > lmax ? lmax : l);
}

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_from(double v)
{
    DF r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

// c j - m for c = tl (uh + ul) (tl a small integer, exact in float), in double-float.
// Every product and sum is rounded explicitly (no contraction into FMA) so the
// error-free transformations stay exact.
__device__ __forceinline__ DF df_step(float tl, float uh, float ul, DF j, DF m)
{
    // coefficient c = ch + cl
    const float ch = __fmul_rn(tl, uh);
    const float cl = fmaf(tl, ul, fmaf(tl, uh, -ch));
    // product p = c j = ph + pl
    const float ph = __fmul_rn(ch, j.hi);
    const float pl = fmaf(ch, j.lo, fmaf(cl, j.hi, fmaf(ch, j.hi, -ph)));
    // two-sum of ph and -m.hi
    const float s = __fsub_rn(ph, m.hi);
    const float v = __fsub_rn(s, ph);
    const float e = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, v)), __fsub_rn(-m.hi, v));
    const float lo = __fsub_rn(__fadd_rn(e, pl), m.lo);
    // renormalise
    DF r;
    r.hi = __fadd_rn(s, lo);
    r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ float series_sum_f(const float *ser, int l, float z)
{
    float s = 1.0f;
#pragma unroll
    for (int n = 7; n >= 1; n--) s = fmaf(-z * ser[8 * l + n], s, 1.0f);
    return s;
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v)
{
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

template <int O>
__device__ __forceinline__ void butterfly_stage_f(float *v, int lane)
{
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; i++) {
        const float send = up ? v[i] : v[i + O];
        const float keep = up ? v[i + O] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

__global__ void __launch_bounds__(32)
project_mixed_kernel(int B, int Nk, const double *__restrict__ bg, long bg_len, const double *__restrict__ S,
                     const double *__restrict__ kv, int lmax, double scale_pol, float *__restrict__ Delta)
{
    extern __shared__ float acc[]; // [2][lmax - 1][2]: Kahan sums, then compensations
    const int nl = lmax - 1;
    float *sum = acc, *comp = acc + 2 * nl;
    ABCMB_CTA_SHARED float ser[8 * kSerL];
    const int blk = blockIdx.x;
    const int kidx = Nk - 1 - blk / B; // high k first
    const int b = blk % B;
    const double *rec = bg + (long)b * bg_len;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    const double tau0 = rec[ABCMB_S_TAU0];
    const double *nodes = rec + ABCMB_BG_NODES;
    const double *Sm = S + ((long)b * Nk + kidx) * (long)n_tau * 3;
    const double kk = kv[kidx];
    const int lane = threadIdx.x;
    for (int i = lane; i < 4 * nl; i += 32) acc[i] = 0.0f;
    for (int i = lane; i < 8 * kSerL; i += 32) {
        const int l = i >> 3, n = i & 7;
        ser[i] = n == 0 ? 1.0f / (2.0f * l + 3.0f) : 1.0f / (2.0f * n * (2.0f * l + 2.0f * n + 1.0f));
    }
    __syncwarp();

    const int gsize = 32 * kNodesPerLane;
    const int ngroups = (n_tau + gsize - 1) / gsize;
    const double s6 = 2.449489742783178; // sqrt(6)
    for (int g = 0; g < ngroups; g++) {
        float A0[kNodesPerLane], A1[kNodesPerLane], A2[kNodesPerLane], Bc[kNodesPerLane], E[kNodesPerLane];
        float uh[kNodesPerLane], ul[kNodesPerLane], t[kNodesPerLane], xs[kNodesPerLane];
        DF jm[kNodesPerLane], jc[kNodesPerLane];
        int lc[kNodesPerLane];
        bool sm[kNodesPerLane];
        int lcmax = 0;
#pragma unroll
        for (int m = 0; m < kNodesPerLane; m++) {
            const int i = g * gsize + m * 32 + lane;
            if (i < n_tau) {
                const double *nd = nodes + 8 * i;
                const double w = nd[N_W];
                const double x = kk * (tau0 - nd[N_TAU]);
                const double u = 1.0 / x;
                const double s0 = Sm[3 * i], s1 = Sm[3 * i + 1], sp = Sm[3 * i + 2];
                const double s2 = scale_pol * sp;
                const double g1 = s1 - 3.0 * u * s2;
                const double u2 = u * u;
                A0[m] = (float)(w * (s0 - s2 - g1 * u));
                A1[m] = (float)(w * (1.5 * s2 * u2 - g1 * u));
                A2[m] = (float)(w * (1.5 * s2 * u2));
                Bc[m] = (float)(w * g1);
                E[m] = (float)(w * s6 * sp * u2);
                const DF ud = df_from(u);
                uh[m] = ud.hi;
                ul[m] = ud.lo;
                sm[m] = x < (double)kSeriesX;
                xs[m] = (float)x;
                double j0, j1, j2;
                if (x < 0.1) {
                    const double x2 = x * x;
                    j0 = 1.0 - x2 * (1.0 / 6.0 - x2 * (1.0 / 120.0 - x2 / 5040.0));
                    j1 = x * (1.0 / 3.0 - x2 * (1.0 / 30.0 - x2 * (1.0 / 840.0 - x2 / 45360.0)));
                } else {
                    double sx, cx;
                    sincos(x, &sx, &cx);
                    j0 = sx * u;
                    j1 = (sx * u - cx) * u;
                }
                j2 = 3.0 * u * j1 - j0;
                if (sm[m]) {
                    const float pf = (float)(x * x / 15.0);
                    t[m] = pf;
                    j2 = (double)(pf * series_sum_f(ser, 2, xs[m] * xs[m]));
                } else {
                    t[m] = 0.0f;
                }
                jm[m] = df_from(j1);
                jc[m] = df_from(j2);
                lc[m] = bessel_cut_f((float)x, lmax);
                if (sm[m] && lc[m] > kSerL - 2) lc[m] = kSerL - 2;
            } else {
                A0[m] = A1[m] = A2[m] = Bc[m] = E[m] = 0.0f;
                uh[m] = ul[m] = t[m] = xs[m] = 0.0f;
                jm[m] = jc[m] = DF{0.0f, 0.0f};
                sm[m] = false;
                lc[m] = 0;
            }
            lcmax = max(lcmax, lc[m]);
        }
        lcmax = __reduce_max_sync(0xffffffffu, lcmax);
        bool anysm = false;
#pragma unroll
        for (int m = 0; m < kNodesPerLane; m++) anysm |= sm[m];
        anysm = __any_sync(0xffffffffu, anysm);
        for (int l0 = 2; l0 <= lcmax + 1 && l0 <= lmax; l0 += kLB) {
            float v[2 * kLB];
            float lf = (float)l0;
#pragma unroll
            for (int q = 0; q < kLB; q++) {
                float cT = 0.0f, cE = 0.0f;
                const int l = l0 + q, lnext = l + 1;
                const float tl = fmaf(2.0f, lf, 1.0f); // 2l + 1, exact
#pragma unroll
                for (int m = 0; m < kNodesPerLane; m++) {
                    const float coef = fmaf(fmaf(A2[m], lf, A1[m]), lf, A0[m]);
                    cT = fmaf(coef, jc[m].hi, cT);
                    cT = fmaf(Bc[m], jm[m].hi, cT);
                    cE = fmaf(E[m], jc[m].hi, cE);
                    DF jn;
                    if (anysm && sm[m]) {
                        const int ls = min(lnext, kSerL - 1);
                        t[m] *= xs[m] * ser[8 * min(l, kSerL - 1)];
                        jn.hi = t[m] * series_sum_f(ser, ls, xs[m] * xs[m]);
                        jn.lo = 0.0f;
                    } else {
                        jn = df_step(tl, uh[m], ul[m], jc[m], jm[m]);
                    }
                    jm[m] = jc[m];
                    const bool keep = lnext <= lc[m];
                    jc[m].hi = keep ? jn.hi : 0.0f;
                    jc[m].lo = keep ? jn.lo : 0.0f;
                }
                v[q] = cT;
                v[kLB + q] = cE;
                lf += 1.0f;
            }
            butterfly_stage_f<16>(v, lane);
            butterfly_stage_f<8>(v, lane);
            butterfly_stage_f<4>(v, lane);
            butterfly_stage_f<2>(v, lane);
            butterfly_stage_f<1>(v, lane);
            const int l = l0 + (lane & (kLB - 1));
            if (l <= lmax) {
                const int idx = 2 * (l - 2) + (lane >> 4);
                kahan_add(sum[idx], comp[idx], v[0]);
            }
            __syncwarp();
        }
    }
    __syncwarp();
    float *out = Delta + ((long)b * Nk + kidx) * (long)nl * 2;
    for (int q = lane; q < nl; q += 32) {
        const double l = q + 2.0;
        const float cE = (float)sqrt(3.0 * (l + 2.0) * (l + 1.0) * l * (l - 1.0) / 8.0);
        out[2 * q] = sum[2 * q];
        out[2 * q + 1] = cE * sum[2 * q + 1];
    }
}

// C_l^{XY} = 4 pi sum_k w_k A_s (k/k_pivot)^(n_s - 1) Delta_X Delta_Y in FP32
// with Kahan-compensated sums; grid (ceil(nl/256), B).
__global__ void cl_mixed_kernel(int B, int Nk, const double *__restrict__ bg, long bg_len,
                                const float *__restrict__ Delta, const double *__restrict__ kv, int lmax,
                                double *__restrict__ Cl)
{
    extern __shared__ float wkf[]; // [Nk]
    const int b = blockIdx.y, nl = lmax - 1;
    const double *rec = bg + (long)b * bg_len;
    const double As = rec[ABCMB_S_AS], ns = rec[ABCMB_S_NS];
    for (int i = threadIdx.x; i < Nk; i += blockDim.x) {
        const double lo = log(kv[i > 0 ? i - 1 : i]), hi = log(kv[i < Nk - 1 ? i + 1 : i]);
        wkf[i] = (float)(4.0 * kPi * 0.5 * (hi - lo) * As * exp((ns - 1.0) * log(kv[i] / kKpivot)));
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nl) return;
    float s[3] = {0.0f, 0.0f, 0.0f}, c[3] = {0.0f, 0.0f, 0.0f};
    const float *D = Delta + (long)b * Nk * nl * 2 + 2 * q;
    for (int i = 0; i < Nk; i++) {
        const float2 d = *reinterpret_cast<const float2 *>(D + (long)i * nl * 2);
        const float f = wkf[i];
        const float fx = __fmul_rn(f, d.x);
        const float term[3] = {__fmul_rn(fx, d.x), __fmul_rn(fx, d.y), __fmul_rn(__fmul_rn(f, d.y), d.y)};
#pragma unroll
        for (int t = 0; t < 3; t++) kahan_add(s[t], c[t], term[t]);
    }
    for (int t = 0; t < 3; t++) Cl[((long)b * 3 + t) * nl + q] = (double)s[t];
}

} // namespace mixed

} // namespace abcmb
