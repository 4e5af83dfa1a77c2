// CMB lensing of the spectra (App. B.5): the all-sky correlation-function
// method the paper cites (Challinor & Lewis 2005), integrated over the whole
// of mu = cos(beta) in [-1, 1] on Gauss-Legendre nodes.  Host+device: the
// kernels in abcmb_lensing.cu call these per node; the CPU tests run them on
// the host.
//
// At each node mu the lensing potential's spectrum gives
//   C_gl(mu)   = sum_l (2l+1)/(4 pi) l(l+1) C^psi_l d^l_11(mu),
//   C_gl,2(mu) = sum_l (2l+1)/(4 pi) l(l+1) C^psi_l d^l_1-1(mu),
//   sigma^2 = C_gl(1) - C_gl(mu),
// and the lensed-minus-unlensed correlation functions xi_T, xi_+, xi_-, xi_x
// are sums over l of the unlensed C_l times Wigner functions d^l_mn(mu) and
// the factors X_imn = exp(-(l(l+1) - c) sigma^2 / 4) (times l-dependent
// roots) of the method, to second order in C_gl,2.  The spectra's changes
// follow by 2 pi sum_nodes w xi d^l_mn with d^l_00, d^l_22, d^l_2-2, d^l_20.
//
// Wigner functions d^l_mn (d^l_mn(0) = delta_mn, d^1_10 = -sin(beta)/sqrt 2)
// start at l = max(|m|, |n|) from the explicit sum over s and rise by the
// three-term recurrence in l; the exponentials by the recurrence
// X(l+1) = X(l) e^{-(l+1) sigma^2 / 2}.
#pragma once

#include <math.h>

#include "abcmb_interp.cuh"

#ifndef ABCMB_HD
#ifdef __CUDACC__
#define ABCMB_HD __host__ __device__ inline
#else
#define ABCMB_HD inline
#endif
#endif

namespace abcmb {
namespace lens {

constexpr double kPi = 3.14159265358979323846;

ABCMB_HD double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

// d^j_mn at j = max(|m|, |n|) from the explicit sum; c = cos(beta/2), s = sin(beta/2)
ABCMB_HD double d_start(int j, int m, int n, double c, double s)
{
    double tot = 0.0;
    for (int k = 0; k <= 2 * j; k++) {
        const int a = j + n - k, b = k, cc = m - n + k, dd = j - m - k;
        if (a < 0 || b < 0 || cc < 0 || dd < 0) continue;
        const double coef = ((m - n + k) % 2 == 0 ? 1.0 : -1.0) *
                            sqrt(fact(j + m) * fact(j - m) * fact(j + n) * fact(j - n)) /
                            (fact(a) * fact(b) * fact(cc) * fact(dd));
        tot += coef * pow(c, 2 * j + n - m - 2 * k) * pow(s, m - n + 2 * k);
    }
    return tot;
}

// one d^l_mn sequence in l: cur = d^l, prv = d^{l-1}
struct DSeq {
    int m, n, j;
    double prv, cur;
};

ABCMB_HD DSeq dseq_init(int m, int n, double mu)
{
    DSeq d;
    d.m = m;
    d.n = n;
    const int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
    d.j = am > an ? am : an;
    const double c = sqrt(fmax(0.5 * (1.0 + mu), 0.0)), s = sqrt(fmax(0.5 * (1.0 - mu), 0.0));
    d.prv = 0.0;
    d.cur = d_start(d.j, m, n, c, s);
    return d;
}

// the value at l (0 below j); advance() moves cur from d^l to d^{l+1} given l
ABCMB_HD double dval(const DSeq &d, int l) { return l < d.j ? 0.0 : d.cur; }

ABCMB_HD void dadvance(DSeq &d, int l, double mu)
{
    if (l < d.j) return;
    const double m = d.m, n = d.n, L = l;
    double nxt;
    if (l == 0) {
        nxt = mu * d.cur; // j = 0: d^1_00 = mu
    } else {
        double num = (2.0 * L + 1.0) * (L * (L + 1.0) * mu - m * n) * d.cur;
        if (l > d.j) num -= (L + 1.0) * sqrt((L * L - m * m) * (L * L - n * n)) * d.prv;
        nxt = num / (L * sqrt(((L + 1.0) * (L + 1.0) - m * m) * ((L + 1.0) * (L + 1.0) - n * n)));
    }
    d.prv = d.cur;
    d.cur = nxt;
}

// unlensed spectra for l = 2..L: tt[l - 2] etc.
struct LensIn {
    const double *tt, *ee, *te, *psi;
    int L;
};

// C_gl(1) = sum (2l+1)/(4 pi) l(l+1) C^psi_l
ABCMB_HD double cgl_at_one(const LensIn &in)
{
    double s = 0.0;
    for (int l = 2; l <= in.L; l++) s += (2.0 * l + 1.0) / (4.0 * kPi) * l * (l + 1.0) * in.psi[l - 2];
    return s;
}

// lensed-minus-unlensed correlation functions at mu: x[0] T, x[1] +, x[2] -, x[3] cross
ABCMB_HD void corr_at(double mu, const LensIn &in, double cgl1, double x[4])
{
    double Cgl = 0.0, G = 0.0;
    {
        DSeq d11 = dseq_init(1, 1, mu), d1m1 = dseq_init(1, -1, mu);
        for (int l = 0; l <= in.L; l++) {
            if (l >= 2) {
                const double f = (2.0 * l + 1.0) / (4.0 * kPi) * l * (l + 1.0) * in.psi[l - 2];
                Cgl += f * dval(d11, l);
                G += f * dval(d1m1, l);
            }
            dadvance(d11, l, mu);
            dadvance(d1m1, l, mu);
        }
    }
    const double sig2 = cgl1 - Cgl;
    DSeq d00 = dseq_init(0, 0, mu), d1m1 = dseq_init(1, -1, mu), d2m2 = dseq_init(2, -2, mu);
    DSeq d22 = dseq_init(2, 2, mu), d31 = dseq_init(3, 1, mu), d40 = dseq_init(4, 0, mu);
    DSeq d3m3 = dseq_init(3, -3, mu), d4m4 = dseq_init(4, -4, mu), d20 = dseq_init(2, 0, mu);
    DSeq d11 = dseq_init(1, 1, mu), d3m1 = dseq_init(3, -1, mu), dm24 = dseq_init(-2, 4, mu);
    // X000(l) = exp(-l(l+1) sigma^2 / 4) by recurrence, and the shifted exponentials
    double X = 1.0;                       // l = 0
    const double e2 = exp(2.0 * sig2 / 4.0), e4 = exp(4.0 * sig2 / 4.0), e83 = exp((8.0 / 3.0) * sig2 / 4.0);
    const double e203 = exp((20.0 / 3.0) * sig2 / 4.0), e10 = exp(10.0 * sig2 / 4.0);
    const double step = exp(-sig2 / 2.0);
    double stepl = 1.0;                   // exp(-(l+1) sigma^2 / 2) at l: starts at l = 0 with e^{-sigma^2/2}
    double xT = 0.0, xP = 0.0, xM = 0.0, xX = 0.0;
    for (int l = 0; l <= in.L; l++) {
        if (l >= 2) {
            const double L = l, lp = L * (L + 1.0), pre = (2.0 * L + 1.0) / (4.0 * kPi);
            const double X000 = X, Xp000 = -lp / 4.0 * X000;
            const double X220 = 0.25 * sqrt(fmax((L + 2.0) * (L - 1.0) * L * (L + 1.0), 0.0)) * X * e2;
            const double X022 = X * e4, Xp022 = -(lp - 4.0) / 4.0 * X022;
            const double X121 = -0.5 * sqrt(fmax((L + 2.0) * (L - 1.0), 0.0)) * X * e83;
            const double X132 = -0.5 * sqrt(fmax((L + 3.0) * (L - 2.0), 0.0)) * X * e203;
            const double X242 = 0.25 * sqrt(fmax((L + 4.0) * (L + 3.0) * (L - 2.0) * (L - 3.0), 0.0)) * X * e10;
            const double tt = in.tt[l - 2], ee = in.ee[l - 2], te = in.te[l - 2];
            xT += pre * tt * ((X000 * X000 - 1.0) * dval(d00, l) + 8.0 / lp * G * Xp000 * Xp000 * dval(d1m1, l) +
                              G * G * (Xp000 * Xp000 * dval(d00, l) + X220 * X220 * dval(d2m2, l)));
            xP += pre * ee * ((X022 * X022 - 1.0) * dval(d22, l) + 2.0 * G * X132 * X121 * dval(d31, l) +
                              G * G * (Xp022 * Xp022 * dval(d22, l) + X242 * X220 * dval(d40, l)));
            xM += pre * ee * ((X022 * X022 - 1.0) * dval(d2m2, l) +
                              G * (X121 * X121 * dval(d1m1, l) + X132 * X132 * dval(d3m3, l)) +
                              0.5 * G * G * (2.0 * Xp022 * Xp022 * dval(d2m2, l) + X220 * X220 * dval(d00, l) +
                                             X242 * X242 * dval(d4m4, l)));
            xX += pre * te * ((X022 * X000 - 1.0) * dval(d20, l) +
                              G * 2.0 * Xp000 / sqrt(lp) * (X121 * dval(d11, l) + X132 * dval(d3m1, l)) +
                              0.5 * G * G * ((2.0 * Xp022 * Xp000 + X220 * X220) * dval(d20, l) +
                                             X220 * X242 * dval(dm24, l)));
        }
        dadvance(d00, l, mu);
        dadvance(d1m1, l, mu);
        dadvance(d2m2, l, mu);
        dadvance(d22, l, mu);
        dadvance(d31, l, mu);
        dadvance(d40, l, mu);
        dadvance(d3m3, l, mu);
        dadvance(d4m4, l, mu);
        dadvance(d20, l, mu);
        dadvance(d11, l, mu);
        dadvance(d3m1, l, mu);
        dadvance(dm24, l, mu);
        // X000(l+1) = X000(l) exp(-(l+1) sigma^2 / 2)
        stepl = l == 0 ? step : stepl * step;
        X *= stepl;
    }
    x[0] = xT;
    x[1] = xP;
    x[2] = xM;
    x[3] = xX;
}

// i-th of n Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n)
ABCMB_HD void gauss_legendre(int n, int i, double *x, double *w)
{
    double z = cos(kPi * (i + 0.75) / (n + 0.5)), pp = 1.0;
    for (int it = 0; it < 100; it++) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; j++) {
            const double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        const double z1 = z;
        z = z1 - p1 / pp;
        if (fabs(z - z1) < 1e-15) break;
    }
    *x = z;
    *w = 2.0 / ((1.0 - z * z) * pp * pp);
}

// ---- the lensing potential in the Limber approximation (App. B.5) ----
//   C_l^psi = 8 pi^2 / (l+1/2)^3 int_0^chi* dchi / chi P_psi((l+1/2)/chi, tau0 - chi) ((chi* - chi)/chi*)^2,
//   P_psi(k, a) = 9 Omega_m(a)^2 H^4 / (8 pi^2 k) P(k, a),
//   P(k, a) = (2 pi^2 / k^3) A_s (k/k_pivot)^(n_s-1) delta_m(k, a)^2,
// on the tau nodes from the visibility peak (chi*) to tau0: the trapezoid
// weights in chi, Omega_m(a) = Omega_m0 H0^2 / (a H^2), delta_m interpolated
// in ln k (lnk_hermite_weights) and zero outside the k nodes.

// node i (8 doubles: ln a, tau, w, g, g', e^-kappa, H, H'); fills chi[i] and
// coef[i] = w_chi / chi 9 Omega_m^2 H^4 / (8 pi^2) ((chi* - chi)/chi*)^2 for
// i >= i_star (the visibility peak), returns i_star
ABCMB_HD int limber_prepare(const double *nodes, int n_tau, double tau0, double Om_m, double H0, double *chi,
                            double *coef)
{
    int is = 0;
    for (int i = 1; i < n_tau; i++)
        if (nodes[8 * i + 3] > nodes[8 * is + 3]) is = i;
    const double chi_star = tau0 - nodes[8 * is + 1];
    for (int i = is; i < n_tau; i++) {
        const double tau = nodes[8 * i + 1], a = exp(nodes[8 * i]), hc = nodes[8 * i + 6];
        const double lo = i > is ? nodes[8 * (i - 1) + 1] : tau, hi = i < n_tau - 1 ? nodes[8 * (i + 1) + 1] : tau0;
        const double c = tau0 - tau, om = Om_m * H0 * H0 / (a * hc * hc), r = (chi_star - c) / chi_star;
        chi[i] = c;
        coef[i] = 0.5 * (hi - lo) / c * 9.0 * om * om * hc * hc * hc * hc / (8.0 * kPi * kPi) * r * r;
    }
    return is;
}

// C_l^psi from delta_m[k][n_tau] at the nodes kv[0..Nk) (Nk >= 4)
ABCMB_HD double limber_cl_at(int l, const double *chi, const double *coef, int i_star, int n_tau, const double *dm,
                             const double *kv, int Nk, double As, double ns)
{
    const double lh = l + 0.5;
    double sum = 0.0;
    for (int i = i_star; i < n_tau; i++) {
        const double k = lh / chi[i];
        if (!(k >= kv[0] && k <= kv[Nk - 1])) continue;
        int r0;
        double w[4];
        lnk_hermite_weights(kv, Nk, k, &r0, w);
        double d = 0.0;
        for (int m = 0; m < 4; m++) d += w[m] * dm[(long)(r0 + m) * n_tau + i];
        const double P = 2.0 * kPi * kPi / (k * k * k) * As * exp((ns - 1.0) * log(k / 0.05)) * d * d;
        sum += coef[i] * P / k;
    }
    return 8.0 * kPi * kPi / (lh * lh * lh) * sum;
}

} // namespace lens
} // namespace abcmb
