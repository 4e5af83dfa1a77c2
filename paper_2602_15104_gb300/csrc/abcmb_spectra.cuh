// Line-of-sight projection and k-quadrature kernels (arXiv 2602.15104,
// App. B.4 transfer functions and eq. c_ell_def; App. B.6 trapezoid rules).
//
// abcmb_project: one CTA per (cosmology, k).  A warp takes groups of
// 32 x kNodesPerLane tau nodes; each lane carries kNodesPerLane independent
// spherical-Bessel recurrences j_{l+1} = (2l+1)/x j_l - j_{l-1} upward in l
// from j_0 = sin x/x, j_1 (power series for x < 1), stopping per node where
// the Debye decay exponent of j_l passes 16 (bessel_cut), which is also where
// the upward recursion would start to lose accuracy.  The coefficient
// (2l+1)/x is formed afresh at every l: accumulated by repeated addition its
// rounding errors would excite the growing solution y_l past the turning
// point and cost several digits there.  With u = 1/x the three temperature kernels collapse to
//   S_T0 j + S_T1 j' + s_pol S_P (3 j'' + j)/2
//     = (A0 + l A1 + l^2 A2) j_l + B j_{l-1},
//   g1 = S_T1 - 3 u s_pol S_P,  A0 = S_T0 - s_pol S_P - g1 u,
//   A1 = 1.5 s_pol S_P u^2 - g1 u,  A2 = 1.5 s_pol S_P u^2,  B = g1
// (from j' = j_{l-1} - (l+1) u j and j'' = -2u j' - (1 - l(l+1)u^2) j), and
// the E kernel to E j_l with E = sqrt(6) S_P u^2 and the l-only factor
// sqrt(3 (l+2)!/(8 (l-2)!)) applied once per l at the end.  Per (node, l):
// 7 FP64 operations.  Lane partial sums for 16 consecutive l (T and E) are
// reduce-scattered across the warp by a 5-stage butterfly and added into the
// CTA's shared Delta[l][2].
#pragma once

#include <math.h>

#include "abcmb_bg.cuh"
#include "abcmb_bessel.cuh"
#include "abcmb_interp.cuh"

namespace abcmb {

constexpr int kNodesPerLane = 4;
constexpr int kLB = 16; // l per block (2 * kLB = 32 partial sums per lane)
// Below x = kSeriesX, j_l comes from its power series
//   j_l(x) = x^l / (2l+1)!! sum_n (-x^2/2)^n / (n! (2l+3)...(2l+2n+1)),
// seven terms (error < 1e-13 for x < 1); ser[8 l] = 1/(2l+3) advances the
// prefactor, ser[8 l + n] = 1 / (2n (2l+2n+1)) is the term ratio.
constexpr double kSeriesX = 1.0;
constexpr int kSerL = 32;

__device__ __forceinline__ double series_sum(const double *ser, int l, double z)
{
    double s = 1.0;
#pragma unroll
    for (int n = 7; n >= 1; n--) s = fma(-z * ser[8 * l + n], s, 1.0);
    return s;
}

__device__ __forceinline__ void j01(double x, double *j0, double *j1)
{
    if (x < 0.1) {
        double x2 = x * x;
        *j0 = 1.0 - x2 * (1.0 / 6.0 - x2 * (1.0 / 120.0 - x2 / 5040.0));
        *j1 = x * (1.0 / 3.0 - x2 * (1.0 / 30.0 - x2 * (1.0 / 840.0 - x2 / 45360.0)));
    } else {
        double s, c;
        sincos(x, &s, &c);
        double u = 1.0 / x;
        *j0 = s * u;
        *j1 = (s * u - c) * u;
    }
}

// One butterfly stage: lanes with bit O set keep the upper half of v[0, 2O)
// and receive the partner's upper-half copy of their kept half.
template <int O>
__device__ __forceinline__ void butterfly_stage(double *v, int lane)
{
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < O; i++) {
        const double send = up ? v[i] : v[i + O];
        const double keep = up ? v[i + O] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// INTERP: the transfer functions at the wavenumbers kv[0..Nk) from sources
// given at the ODE nodes kode[0..Nko) (S[B][Nko][n_tau][3]), interpolated per
// node in ln k (lnk_hermite_weights); otherwise S is given at kv itself.
template <bool INTERP>
__global__ void __launch_bounds__(128)
project_kernel(int B, int Nk, const double *__restrict__ bg, long bg_len,
               const double *__restrict__ S, const double *__restrict__ kv, int lmax,
               double scale_pol, double *__restrict__ Delta, const double *__restrict__ kode, int Nko)
{
    extern __shared__ double acc[]; // [lmax - 1][2]
    const int nl = lmax - 1;
    const int blk = blockIdx.x;
    const int kidx = Nk - 1 - blk / B; // high k first
    const int b = blk % B;
    const double *rec = bg + (long)b * bg_len;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    const double tau0 = rec[ABCMB_S_TAU0];
    const double *nodes = rec + ABCMB_BG_NODES;
    const double kk = kv[kidx];
    const double *Sm;
    int r0 = 0;
    double wi[4] = {0.0, 0.0, 0.0, 0.0};
    long rs = 0; // element stride between consecutive source rows
    if (INTERP) {
        lnk_hermite_weights(kode, Nko, kk, &r0, wi);
        Sm = S + ((long)b * Nko + r0) * (long)n_tau * 3;
        rs = (long)n_tau * 3;
    } else {
        Sm = S + ((long)b * Nk + kidx) * (long)n_tau * 3;
    }
    ABCMB_CTA_SHARED double ser[8 * kSerL];
    for (int i = threadIdx.x; i < 2 * nl; i += blockDim.x) acc[i] = 0.0;
    for (int i = threadIdx.x; i < 8 * kSerL; i += blockDim.x) {
        const int l = i >> 3, n = i & 7;
        ser[i] = n == 0 ? 1.0 / (2.0 * l + 3.0) : 1.0 / (2.0 * n * (2.0 * l + 2.0 * n + 1.0));
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int gsize = 32 * kNodesPerLane;
    const int ngroups = (n_tau + gsize - 1) / gsize;
    const double s6 = 2.449489742783178; // sqrt(6)
    for (int g = warp; g < ngroups; g += W) {
        double A0[kNodesPerLane], A1[kNodesPerLane], A2[kNodesPerLane], Bc[kNodesPerLane], E[kNodesPerLane];
        double jm[kNodesPerLane], jc[kNodesPerLane], t[kNodesPerLane], tu[kNodesPerLane];
        // nodes with x < kSeriesX keep x^l/(2l+1)!! in t[] and x in tu[]
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
                double s0, s1, sp;
                if (INTERP) {
                    s0 = s1 = sp = 0.0;
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const double *Sr = Sm + r * rs + 3 * i;
                        s0 = fma(wi[r], Sr[0], s0);
                        s1 = fma(wi[r], Sr[1], s1);
                        sp = fma(wi[r], Sr[2], sp);
                    }
                } else {
                    s0 = Sm[3 * i];
                    s1 = Sm[3 * i + 1];
                    sp = Sm[3 * i + 2];
                }
                const double s2 = scale_pol * sp;
                const double g1 = s1 - 3.0 * u * s2;
                const double u2 = u * u;
                A0[m] = w * (s0 - s2 - g1 * u);
                A1[m] = w * (1.5 * s2 * u2 - g1 * u);
                A2[m] = w * (1.5 * s2 * u2);
                Bc[m] = w * g1;
                E[m] = w * s6 * sp * u2;
                double j0, j1;
                j01(x, &j0, &j1);
                jm[m] = j1;
                sm[m] = x < kSeriesX;
                jc[m] = sm[m] ? x * x / 15.0 * series_sum(ser, 2, x * x) : 3.0 * u * j1 - j0; // j_2
                t[m] = sm[m] ? x * x / 15.0 : 0.0;
                tu[m] = sm[m] ? x : u;
                lc[m] = bessel_cut((float)x, lmax);
                if (sm[m] && lc[m] > kSerL - 2) lc[m] = kSerL - 2;
            } else {
                A0[m] = A1[m] = A2[m] = Bc[m] = E[m] = 0.0;
                jm[m] = jc[m] = t[m] = tu[m] = 0.0;
                sm[m] = false;
                lc[m] = 0;
            }
            lcmax = max(lcmax, lc[m]);
        }
        lcmax = __reduce_max_sync(0xffffffffu, lcmax);
        bool anysm = false;
#pragma unroll
        for (int m = 0; m < kNodesPerLane; m++) anysm |= sm[m];
        anysm = __any_sync(0xffffffffu, anysm); // warp-uniform
        // past its cutoff a node's j is held at exactly zero (the upward
        // recurrence is unstable there), so it contributes nothing further
        for (int l0 = 2; l0 <= lcmax + 1 && l0 <= lmax; l0 += kLB) {
            double v[2 * kLB];
            double ld = (double)l0;
            if (!anysm) {
#pragma unroll
                for (int q = 0; q < kLB; q++) {
                    double cT = 0.0, cE = 0.0;
                    const int lnext = l0 + q + 1;
                    const double tl = fma(2.0, ld, 1.0); // 2l + 1, exact
#pragma unroll
                    for (int m = 0; m < kNodesPerLane; m++) {
                        const double coef = fma(fma(A2[m], ld, A1[m]), ld, A0[m]);
                        cT = fma(coef, jc[m], cT);
                        cT = fma(Bc[m], jm[m], cT);
                        cE = fma(E[m], jc[m], cE);
                        const double jn = fma(tl * tu[m], jc[m], -jm[m]);
                        jm[m] = jc[m];
                        jc[m] = lnext <= lc[m] ? jn : 0.0;
                    }
                    v[q] = cT;
                    v[kLB + q] = cE;
                    ld += 1.0;
                }
            } else {
                // some node of the group has x < 1: those take j_{l+1} from
                // its power series instead of the (there unstable) recurrence
#pragma unroll
                for (int q = 0; q < kLB; q++) {
                    double cT = 0.0, cE = 0.0;
                    const int l = l0 + q, lnext = l + 1;
                    const int ls = min(lnext, kSerL - 1);
                    const double tl = fma(2.0, ld, 1.0);
#pragma unroll
                    for (int m = 0; m < kNodesPerLane; m++) {
                        const double coef = fma(fma(A2[m], ld, A1[m]), ld, A0[m]);
                        cT = fma(coef, jc[m], cT);
                        cT = fma(Bc[m], jm[m], cT);
                        cE = fma(E[m], jc[m], cE);
                        double jn;
                        if (sm[m]) {
                            t[m] *= tu[m] * ser[8 * min(l, kSerL - 1)];
                            jn = t[m] * series_sum(ser, ls, tu[m] * tu[m]);
                        } else {
                            jn = fma(tl * tu[m], jc[m], -jm[m]);
                        }
                        jm[m] = jc[m];
                        jc[m] = lnext <= lc[m] ? jn : 0.0;
                    }
                    v[q] = cT;
                    v[kLB + q] = cE;
                    ld += 1.0;
                }
            }
            // reduce-scatter: lane ends with the warp total of v[lane]
            butterfly_stage<16>(v, lane);
            butterfly_stage<8>(v, lane);
            butterfly_stage<4>(v, lane);
            butterfly_stage<2>(v, lane);
            butterfly_stage<1>(v, lane);
            const int l = l0 + (lane & (kLB - 1));
            if (l <= lmax) atomicAdd(&acc[2 * (l - 2) + (lane >> 4)], v[0]);
        }
    }
    __syncthreads();
    double *out = Delta + ((long)b * Nk + kidx) * (long)nl * 2;
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
        const double l = q + 2.0;
        const double cE = sqrt(3.0 * (l + 2.0) * (l + 1.0) * l * (l - 1.0) / 8.0);
        out[2 * q] = acc[2 * q];
        out[2 * q + 1] = cE * acc[2 * q + 1];
    }
}

// C_l^{XY} = 4 pi sum_k w_k A_s (k/k_pivot)^(n_s - 1) Delta_X Delta_Y,
// trapezoid in ln k; compensated (Kahan) sums.  grid (ceil(nl/256), B).
__global__ void cl_kernel(int B, int Nk, const double *__restrict__ bg, long bg_len,
                          const double *__restrict__ Delta, const double *__restrict__ kv,
                          int lmax, double *__restrict__ Cl)
{
    extern __shared__ double wk[]; // [Nk]
    const int b = blockIdx.y, nl = lmax - 1;
    const double *rec = bg + (long)b * bg_len;
    const double As = rec[ABCMB_S_AS], ns = rec[ABCMB_S_NS];
    for (int i = threadIdx.x; i < Nk; i += blockDim.x) {
        double lo = log(kv[i > 0 ? i - 1 : i]), hi = log(kv[i < Nk - 1 ? i + 1 : i]);
        wk[i] = 4.0 * kPi * 0.5 * (hi - lo) * As * exp((ns - 1.0) * log(kv[i] / kKpivot));
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nl) return;
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    const double *D = Delta + (long)b * Nk * nl * 2 + 2 * q;
    for (int i = 0; i < Nk; i++) {
        const double2 d = *reinterpret_cast<const double2 *>(D + (long)i * nl * 2);
        const double f = wk[i];
        const double term[3] = {f * d.x * d.x, f * d.x * d.y, f * d.y * d.y};
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const double y = term[t] - c[t];
            const double tt = s[t] + y;
            c[t] = (tt - s[t]) - y;
            s[t] = tt;
        }
    }
    for (int t = 0; t < 3; t++) Cl[((long)b * 3 + t) * nl + q] = s[t];
}

} // namespace abcmb
