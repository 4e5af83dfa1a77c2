// Per-mode integration of the synchronous-gauge perturbation ODEs and the CMB
// sources at the tau nodes (arXiv 2602.15104, App. B.3.1, App. B.4, App. C).
//
// State (this library's own formulation; photons and neutrinos carried as
// Legendre moments F_l throughout, F_1 = 4 theta / (3k), F_2 = 2 sigma):
//   [eta, delta_c, delta_b, theta_b, F_g0..F_gLg, G_0..G_Lp, F_n0..F_nLn]
// Equations in x = ln a (k_H = k / H_conf), which restate App. C in F_l:
//   h'   = 2 k_H^2 eta + 3 sum f_i delta_i                        (eq. hprime)
//   eta' = (3/2) / k_H (f_b theta_b / k + f_g F_g1 + f_n F_n1)       (eq. etaprime)
//   delta_c' = -h'/2,  delta_b' = -theta_b / H - h'/2
//   theta_b' = -theta_b + c_s^2 k^2 delta_b / H + R^-1 nu (3k/4 F_g1 - theta_b)
//   F_l' = k_H / (2l+1) (l F_{l-1} - (l+1) F_{l+1})  (l < L),
//   F_L' = k_H F_{L-1} - (L+1) / (H tau) F_L                       (truncation)
//   metric terms: F_0' -= 2/3 h',  F_2' += 4/15 h' + 8/5 eta'
//   Thomson (photons only, nu = 1/(H tau_c)):
//     F_g1' += nu (4/(3k) theta_b - F_g1),  F_gl' -= nu F_gl (l >= 2),
//     G_l'  -= nu G_l,  Pi = F_g2 + G_0 + G_2:
//     F_g2' += nu Pi / 10, G_0' += nu Pi / 2, G_2' += nu Pi / 10
// (the -(9/10) sigma and (1/20)(G_0 + G_2) of App. C.4 in F_2 form, and the
// polarization source read as Pi (delta_l0 + delta_l2 / 5) / 2).
//
// Integrator, two regimes (both extrapolation methods, no tableau constants):
//  * while 1/(H tau_c) >= 1 (up to recombination): linearly implicit (IMEX)
//    Euler with the Thomson terms implicit -- they are the only stiff terms
//    and form a 2x2 block (theta_b, F_g1), a rank-one-plus-diagonal 3x3 block
//    (F_g2, G_0, G_2) and a diagonal -- and everything else explicit;
//    Aitken-Neville extrapolation in h over the substep counts 1, 2, ..., K;
//  * afterwards (free streaming, non-stiff): explicit midpoint rule
//    (Gragg) with 2, 4, ..., 2K substeps extrapolated in h^2 (GBS).
// The difference of the two highest orders is the error estimate; a step is
// accepted at the first column that meets the tolerance.  Steps land exactly
// on every tau node, where the sources are evaluated (App. B.4, eq.
// source_functions).
#pragma once

#include "abcmb_bg.cuh"

namespace abcmb {

constexpr int kKmax = 6;    // highest extrapolation column
constexpr int kNvec = kKmax + 2;
// Error scale of component i: atol + rtol max(|y_i|, kChainFloor * m_g), m_g
// the largest magnitude in i's group at the step start; groups: {eta, delta_c,
// delta_b}, {theta_b}, photons {F_g, G} together, neutrinos {F_n}.  Sharing
// the photon group keeps the tiny tight-coupled polarization moments from
// dictating the step in the stiff early era.
#ifndef ABCMB_CHAIN_FLOOR
#define ABCMB_CHAIN_FLOOR 1e-4
#endif
// Explicit Gragg-Bulirsch-Stoer steps once 1/(H tau_c) < kNuNonStiff (after
// recombination); while H 1/(H tau_c) > kSlavedHnu the photon moments l >= 2
// and the polarization moments are slaved to the slow variables (their local
// errors are damped by 1/(1 + h nu) every substep) and leave the error norm.
constexpr double kNuNonStiff = 1.0;
constexpr double kSlavedHnu = 100.0;

struct OdeDims {
    int Lg, Lp, Ln, N;
    int iF, iG, iN; // first index of each chain
    int Lm, iM;     // massive neutrinos: 3 momentum bins of Psi_0..Psi_Lm from iM (Lm = 0: none)
};

ABCMB_HD OdeDims ode_dims(int Lg, int Lp, int Ln, int Lm = 0)
{
    OdeDims d;
    d.Lg = Lg; d.Lp = Lp; d.Ln = Ln; d.Lm = Lm;
    d.iF = 4;
    d.iG = d.iF + Lg + 1;
    d.iN = d.iG + Lp + 1;
    d.iM = d.iN + Ln + 1;
    d.N = d.iM + (Lm > 0 ? 3 * (Lm + 1) : 0);
    return d;
}

// Strided view of one vector of the per-mode working set.
struct Vec {
    double *p;
    long stride;
    ABCMB_HD double &operator[](int i) const { return p[(long)i * stride]; }
};

// Streaming coefficients l/(2l+1) and (l+1)/(2l+1), l = 0..128.
struct StreamCoef {
    const double *a, *b;
};

// One linearly implicit Euler substep of size hs from x_m (background bc,
// explicit terms) to x_{m+1} (background bn, implicit Thomson terms), in place.
ABCMB_HD void imex_substep(const OdeDims &d, const StreamCoef &sc, double k, double hs,
                           const BgPt &bc, const BgPt &bn, Vec y)
{
    const double kH = k * bc.inv_Hc;
    // metric from the state at x_m
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    const double Fg0 = y[d.iF], Fg1 = y[d.iF + 1], Fn0 = y[d.iN], Fn1 = y[d.iN + 1];
    const double hp = 2.0 * kH * kH * eta + 3.0 * (bc.fc * dc + bc.fb * db + bc.fg * Fg0 + bc.fnu * Fn0);
    const double ep = 1.5 / kH * (bc.fb * tb / k + bc.fg * Fg1 + bc.fnu * Fn1);
    // explicit part
    y[0] = eta + hs * ep;
    y[1] = dc - hs * 0.5 * hp;
    y[2] = db + hs * (-tb * bc.inv_Hc - 0.5 * hp);
    y[3] = tb + hs * (-tb + bc.cs2 * k * k * db * bc.inv_Hc);
    const double trunc = bc.inv_Hc / bc.tau;
    const double hpe = hs * (-2.0 / 3.0) * hp, h2e = hs * ((4.0 / 15.0) * hp + 1.6 * ep);
    // three chains; metric terms on F_0 and F_2 of the photon and neutrino chains
    for (int ch = 0; ch < 3; ch++) {
        int i0 = ch == 0 ? d.iF : ch == 1 ? d.iG : d.iN;
        int L = ch == 0 ? d.Lg : ch == 1 ? d.Lp : d.Ln;
        double prev = 0.0;
        for (int l = 0; l < L; l++) {
            double cur = y[i0 + l], nxt = y[i0 + l + 1];
            double v = cur + hs * kH * (sc.a[l] * prev - sc.b[l] * nxt);
            y[i0 + l] = v;
            prev = cur;
        }
        double cur = y[i0 + L];
        y[i0 + L] = cur + hs * (kH * prev - (L + 1.0) * trunc * cur);
        if (ch != 1) {
            y[i0] += hpe;
            y[i0 + 2] += h2e;
        }
    }
    // implicit Thomson part at x_{m+1}
    const double nu = bn.nuT, hnu = hs * nu, dmp = 1.0 / (1.0 + hnu);
    {
        const double hRnu = hs * bn.Rinv * nu;
        const double rb = y[3], ru = 0.75 * k * y[d.iF + 1];
        const double idet = 1.0 / (1.0 + hRnu + hnu);
        y[3] = ((1.0 + hnu) * rb + hRnu * ru) * idet;
        const double un = (hnu * rb + (1.0 + hRnu) * ru) * idet;
        y[d.iF + 1] = un * (4.0 / 3.0) / k;
    }
    {
        const double r2 = y[d.iF + 2], g0 = y[d.iG], g2 = y[d.iG + 2];
        const double pin = (r2 + g0 + g2) / (1.0 + 0.3 * hnu);
        y[d.iF + 2] = (r2 + 0.1 * hnu * pin) * dmp;
        y[d.iG] = (g0 + 0.5 * hnu * pin) * dmp;
        y[d.iG + 2] = (g2 + 0.1 * hnu * pin) * dmp;
    }
    for (int l = 3; l <= d.Lg; l++) y[d.iF + l] *= dmp;
    y[d.iG + 1] *= dmp;
    for (int l = 3; l <= d.Lp; l++) y[d.iG + l] *= dmp;
}


// dst += fac * f(x, src), full right-hand side with the Thomson terms explicit
ABCMB_HD void rhs_axpy(const OdeDims &d, const StreamCoef &sc, double k, const BgPt &b, Vec src, Vec dst,
                       double fac)
{
    const double kH = k * b.inv_Hc;
    const double eta = src[0], dc = src[1], db = src[2], tb = src[3];
    const double Fg0 = src[d.iF], Fg1 = src[d.iF + 1], Fn0 = src[d.iN], Fn1 = src[d.iN + 1];
    const double hp = 2.0 * kH * kH * eta + 3.0 * (b.fc * dc + b.fb * db + b.fg * Fg0 + b.fnu * Fn0);
    const double ep = 1.5 / kH * (b.fb * tb / k + b.fg * Fg1 + b.fnu * Fn1);
    const double nu = b.nuT;
    dst[0] += fac * ep;
    dst[1] += fac * (-0.5 * hp);
    dst[2] += fac * (-tb * b.inv_Hc - 0.5 * hp);
    dst[3] += fac * (-tb + b.cs2 * k * k * db * b.inv_Hc + b.Rinv * nu * (0.75 * k * Fg1 - tb));
    const double trunc = b.inv_Hc / b.tau;
    const double Pi = src[d.iF + 2] + src[d.iG] + src[d.iG + 2];
    for (int ch = 0; ch < 3; ch++) {
        const int i0 = ch == 0 ? d.iF : ch == 1 ? d.iG : d.iN;
        const int L = ch == 0 ? d.Lg : ch == 1 ? d.Lp : d.Ln;
        const double damp = ch == 2 ? 0.0 : nu;
        double prev = 0.0;
        for (int l = 0; l < L; l++) {
            const double cur = src[i0 + l];
            double v = kH * (sc.a[l] * prev - sc.b[l] * src[i0 + l + 1]) - damp * cur;
            dst[i0 + l] += fac * v;
            prev = cur;
        }
        const double cur = src[i0 + L];
        dst[i0 + L] += fac * (kH * prev - (L + 1.0) * trunc * cur - damp * cur);
    }
    // corrections: photon F_0 has no damping, F_1 couples to theta_b, Pi sources
    dst[d.iF] += fac * (nu * Fg0 - (2.0 / 3.0) * hp);
    dst[d.iF + 1] += fac * nu * (4.0 / 3.0) * tb / k;
    dst[d.iF + 2] += fac * (0.1 * nu * Pi + (4.0 / 15.0) * hp + 1.6 * ep);
    dst[d.iG] += fac * 0.5 * nu * Pi;
    dst[d.iG + 2] += fac * 0.1 * nu * Pi;
    dst[d.iN] += fac * (-(2.0 / 3.0) * hp);
    dst[d.iN + 2] += fac * ((4.0 / 15.0) * hp + 1.6 * ep);
}

ABCMB_HD void initial_state(const OdeDims &d, const Cosmo &c, double k, double tau_i, Vec y)
{
    for (int i = 0; i < d.N; i++) y[i] = 0.0;
    const double C = 0.5, Rn = c.R_nu, kt = k * tau_i;
    const double dg = -(2.0 / 3.0) * C * kt * kt;
    const double F1 = -(2.0 / 27.0) * C * kt * kt * kt;          // 4/(3k) theta_g
    const double tg = -C * k * kt * kt * kt / 18.0;
    y[0] = 2.0 * C - C * kt * kt * (5.0 + 4.0 * Rn) / (6.0 * (15.0 + 4.0 * Rn));
    y[1] = 0.75 * dg;
    y[2] = 0.75 * dg;
    y[3] = tg;
    y[d.iF] = dg;
    y[d.iF + 1] = F1;
    y[d.iN] = dg;
    y[d.iN + 1] = F1 * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn);
    y[d.iN + 2] = (8.0 / 3.0) * C * kt * kt / (15.0 + 4.0 * Rn);
}

// Sources at a tau node from the state there (App. B.4, eq. source_functions).
ABCMB_HD void node_sources(const OdeDims &d, const Cosmo &c, const double *tab, const double *nd,
                           double k, const double sw[3], Vec y, double *S)
{
    BgPt b = bg_point(c, tab, nd[N_LNA]);
    const double Hc = nd[N_HC], dHc = nd[N_DHC], g = nd[N_G], dg = nd[N_DG], emk = nd[N_EXPMK];
    const double kH = k / Hc, k2 = k * k;
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    const double Fg0 = y[d.iF], Fg1 = y[d.iF + 1], Fg2 = y[d.iF + 2];
    const double Fn0 = y[d.iN], Fn1 = y[d.iN + 1], Fn2 = y[d.iN + 2];
    const double hp = 2.0 * kH * kH * eta + 3.0 * (b.fc * dc + b.fb * db + b.fg * Fg0 + b.fnu * Fn0);
    const double ep = 1.5 / kH * (b.fb * tb / k + b.fg * Fg1 + b.fnu * Fn1);
    const double alpha = Hc * (hp + 6.0 * ep) / (2.0 * k2);
    const double shear = (2.0 / 3.0) * (b.fg * Fg2 + b.fnu * Fn2); // sum f (1+w) sigma
    const double Hap = -2.0 * Hc * alpha + eta - 4.5 * Hc * Hc / k2 * shear; // H alpha'
    const double ap = Hap / Hc;
    const double tbp = -tb + b.cs2 * k2 * db / Hc + b.Rinv * b.nuT * (0.75 * k * Fg1 - tb);
    const double swt = g * (0.25 * Fg0 + Hap);
    const double isw = g * (eta - Hap - 2.0 * Hc * alpha) + 2.0 * Hc * emk * (ep - dHc * alpha - Hap);
    const double dop = Hc * (g * (tbp / k2 + ap) + dg * (tb / k2 + alpha));
    S[0] = sw[0] * swt + sw[1] * isw + sw[2] * dop;
    S[1] = sw[1] * emk * k * (Hap + 2.0 * Hc * alpha - eta);
    S[2] = g * (Fg2 + y[d.iG] + y[d.iG + 2]) * 0.125;
}

struct ModeResult {
    int status, steps, substeps;
};

// Integrate one (cosmology, k) mode and write S[n_tau][3].
// work: kNvec vectors (Y, YS, T_0..T_{K-1}) of N entries with the given stride.
ABCMB_HD ModeResult integrate_mode(const OdeDims &d, const StreamCoef &sc, const double *rec,
                                   double k, double rtol, double atol, int max_steps,
                                   const double sw[3], double *work, long wstride,
                                   double *S)
{
    ModeResult res = {ABCMB_OK, 0, 0};
    const Cosmo c = load_cosmo(rec);
    const double *tab = rec + ABCMB_BG_TABLE;
    const double *nodes = rec + ABCMB_BG_NODES;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    const long vlen = (long)d.N * wstride;
    Vec Y = {work, wstride}, YS = {work + vlen, wstride};
    Vec T[kKmax];
    for (int j = 0; j < kKmax; j++) T[j] = Vec{work + (2 + j) * vlen, wstride};

    // start: a_i = min(a_tc, a_k), k / H(a_k) = R_large (App. A.1)
    double x = c.lna_tc;
    const double target = k / kRlarge;
    if (hconf(c, c.lna_tc) < target) {
        double lo = kLna0, hi = c.lna_tc;
        if (hconf(c, lo) < target) x = lo;
        else {
            for (int it = 0; it < 100; it++) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                if (hconf(c, mid) > target) lo = mid; else hi = mid;
            }
            x = 0.5 * (lo + hi);
        }
    }
    {
        Herm H = herm_at(x);
        initial_state(d, c, k, herm_val(tab, H, C_TAU, C_DTAU), Y);
    }
    double h = 1e-3;
    int node = 0;
    // non-stiff switch: where 1/(H tau_c) falls below kNuNonStiff after recombination
    double x_ns = 0.0;
    {
        double lo = c.lna_sw, hi = -2.0;
        for (int it = 0; it < 60; it++) {
            double mid = 0.5 * (lo + hi);
            Herm Hm = herm_at(mid);
            if (herm_val(tab, Hm, C_NUT, C_DNUT) > kNuNonStiff) lo = mid; else hi = mid;
        }
        x_ns = hi;
    }
    while (node < n_tau) {
        const double xn = nodes[8 * node + N_LNA];
        double H = h;
        bool land = false;
        if (x + H >= xn) { H = xn - x; land = true; }
        if (H > 0.0) {
            if (++res.steps > max_steps) { res.status = ABCMB_E_MAX_STEPS; break; }
            if (H < 1e-13 && !land) { res.status = ABCMB_E_NONFINITE; break; } // step size underflow
            // per-chain magnitudes for the error scale
            double cm[5] = {0, 0, 0, 0, 0};
            for (int i = 0; i < d.N; i++) {
                int g = i < 3 ? 0 : i == 3 ? 1 : i < d.iN ? 2 : 4;
                double v = fabs(Y[i]);
                if (v > cm[g]) cm[g] = v;
            }
            const BgPt b0 = bg_point(c, tab, x);
            BgPt bend;
            double err = 0.0;
            int jacc = 0;
            const bool gbs = x >= x_ns;
            const bool slaved = H * b0.nuT > kSlavedHnu;
            for (int j = 1; j <= kKmax; j++) {
              if (gbs) {
                const int n = 2 * j;
                const double hs = H / n;
                res.substeps += n;
                for (int i = 0; i < d.N; i++) { YS[i] = Y[i]; T[kKmax - 1][i] = Y[i]; }
                // YS = z0, TK = z1 = z0 + hs f(z0)
                Vec za = YS, zb = T[kKmax - 1];
                rhs_axpy(d, sc, k, b0, za, zb, hs);
                for (int m = 1; m < n; m++) {
                    BgPt bm = bg_point(c, tab, x + m * hs);
                    rhs_axpy(d, sc, k, bm, zb, za, 2.0 * hs);
                    Vec t = za; za = zb; zb = t;
                }
                // z_n is in zb
                err = 0.0;
                for (int i = 0; i < d.N; i++) {
                    double cur = zb[i], prev = T[0][i];
                    T[0][i] = cur;
                    for (int s2 = 1; s2 < j; s2++) {
                        double r = (double)j / (double)(j - s2);
                        double nw = cur + (cur - prev) / (r * r - 1.0);
                        prev = T[s2][i];
                        T[s2][i] = nw;
                        cur = nw;
                    }
                    if (j >= 2) {
                        int g = i < 3 ? 0 : i == 3 ? 1 : i < d.iN ? 2 : 4;
                        double scl = atol + rtol * fmax(fmax(fabs(Y[i]), fabs(T[j - 1][i])), ABCMB_CHAIN_FLOOR * cm[g]);
                        double e = fabs(T[j - 1][i] - T[j - 2][i]) / scl;
                        if (!(e <= err)) err = e;
                    }
                }
                if (!(err == err)) break;
                if (j >= 2 && err <= 1.0) { jacc = j; break; }
                continue;
              }
                const double hs = H / j;
                res.substeps += j;
                for (int i = 0; i < d.N; i++) YS[i] = Y[i];
                BgPt bc = b0;
                for (int m = 0; m < j; m++) {
                    BgPt bn;
                    if (m == j - 1) {
                        if (j == 1) bend = bg_point(c, tab, x + H);
                        bn = bend;
                    } else {
                        bn = bg_point(c, tab, x + (m + 1) * hs);
                    }
                    imex_substep(d, sc, k, hs, bc, bn, YS);
                    bc = bn;
                }
                err = 0.0;
                for (int i = 0; i < d.N; i++) {
                    double cur = YS[i], prev = T[0][i];
                    T[0][i] = cur;
                    for (int s = 1; s < j; s++) {
                        double nw = cur + (cur - prev) * (double)(j - s) / (double)s;
                        prev = T[s][i];
                        T[s][i] = nw;
                        cur = nw;
                    }
                    if (j >= 2 && !(slaved && i >= d.iF + 2 && i < d.iN)) {
                        int g = i < 3 ? 0 : i == 3 ? 1 : i < d.iN ? 2 : 4;
                        double scl = atol + rtol * fmax(fmax(fabs(Y[i]), fabs(T[j - 1][i])),
                                                        ABCMB_CHAIN_FLOOR * cm[g]);
                        double e = fabs(T[j - 1][i] - T[j - 2][i]) / scl;
                        if (!(e <= err)) err = e; // propagates NaN
                    }
                }
                if (!(err == err)) break;
                if (j >= 2 && err <= 1.0) { jacc = j; break; }
            }
            if (!(err == err) || err > 1e300) { res.status = ABCMB_E_NONFINITE; break; }
            if (jacc) {
                for (int i = 0; i < d.N; i++) Y[i] = T[jacc - 1][i];
                x = land ? xn : x + H;
                double fac = err > 0.0 ? 0.9 * exp(-log(err) / (gbs ? 2 * jacc - 1 : jacc)) : 4.0;
                if (jacc < kKmax - 1) fac *= 1.5;
                fac = fmin(4.0, fmax(0.2, fac));
                double hn = H * fac;
                h = land ? fmax(h, hn) : hn;
                if (land) {
                    double sv[3];
                    node_sources(d, c, tab, nodes + 8 * node, k, sw, Y, sv);
                    S[3 * node] = sv[0];
                    S[3 * node + 1] = sv[1];
                    S[3 * node + 2] = sv[2];
                    node++;
                }
            } else {
                double fac = fmin(0.9, fmax(0.1, 0.9 * exp(-log(err) / (gbs ? 2 * kKmax - 1 : kKmax))));
                h = H * fac;
            }
        } else {
            // x already at the node (first node equal to the start time)
            double sv[3];
            node_sources(d, c, tab, nodes + 8 * node, k, sw, Y, sv);
            S[3 * node] = sv[0];
            S[3 * node + 1] = sv[1];
            S[3 * node + 2] = sv[2];
            node++;
        }
    }
    for (int n = node; n < n_tau; n++) S[3 * n] = S[3 * n + 1] = S[3 * n + 2] = 0.0;
    return res;
}

} // namespace abcmb
