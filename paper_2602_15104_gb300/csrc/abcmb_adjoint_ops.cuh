// Linear operators of the perturbation ODE for the discrete adjoint
// (thread-per-mode state layout of abcmb_ode.cuh; background quantities from
// the ODE table of the background record).
//
// The right-hand side y' = (E(b) + T(b)) y is linear in the state y and splits
// into E, everything but Thomson scattering, and T, the Thomson terms (the
// only stiff ones; abcmb_ode.cuh lists both).  For each operator this file
// gives  out += fac X y,  out += fac X^T v  and  bbar += fac d(v^T X(b) y)/db
// for the ten background quantities b, plus the IMEX solve (I - h T)^{-1} and
// its transpose, the CMB sources at a node with their reverse mode, and the
// adiabatic initial state with its derivative in tau_i.  Everything is
// host+device so that the identities <v, X y> = <X^T v, y> and the b-gradients
// can be checked against finite differences on the CPU.
#pragma once

#include "abcmb_ode.cuh"

namespace abcmb {
namespace adj {

// background quantities at one ln a, in ODE-table column order
enum { B_IH = 0, B_IHT, B_FC, B_FB, B_FG, B_FNU, B_NU, B_RNU, B_CS2, B_HC, B_N };

struct Bg10 {
    double v[B_N];
    // massive neutrino at this point (not table columns): x = a m / T_ncdm and
    // nn = PREF a^-4 / (rho_tot / rho_crit), which turns the momentum sums into
    // fractions of rho_tot (both 0 without one)
    double nx = 0.0, nn = 0.0;
};

// Momentum bins of the perturbed massive-neutrino integrals (App. B.3, the
// paper's 3-point rule) and d ln f_0 / d ln q = -q / (1 + e^-q) at them.
ABCMB_HD double ncdm_q(int j) { return j == 0 ? 0.913201 : (j == 1 ? 3.37517 : 7.79184); }
ABCMB_HD double ncdm_k(int j) { return j == 0 ? 0.0687359 : (j == 1 ? 3.31435 : 2.29911); }

// delta rho, (rho + p) theta / k and (rho + p) sigma of the massive neutrinos
// as fractions of rho_tot (eq. mnu_sum); y[d.iM + j (Lm + 1) + l] = Psi_l(q_j)
ABCMB_HD void ncdm_sums(const OdeDims &d, const Bg10 &b, Vec y, double &drho, double &rpth_k, double &rpsig)
{
    drho = rpth_k = rpsig = 0.0;
    if (d.Lm <= 0) return;
    for (int j = 0; j < 3; j++) {
        const double q = ncdm_q(j), eps = sqrt(q * q + b.nx * b.nx), w = ncdm_k(j) * (1.0 + exp(-q));
        const int i0 = d.iM + j * (d.Lm + 1);
        drho += w * eps / (q * q) * y[i0];
        rpth_k += w / q * y[i0 + 1];
        rpsig += (2.0 / 3.0) * w / eps * y[i0 + 2];
    }
    drho *= b.nn;
    rpth_k *= b.nn;
    rpsig *= b.nn;
}

// cubic Hermite on the ODE table (20 doubles per row: value, d/dln a pairs)
struct HW {
    int j;
    double w0, w1, d0, d1;
};

ABCMB_HD HW hw_at(double lna)
{
    HW h;
    const double t = (lna - kLna0) * ABCMB_BG_PER_UNIT;
    int j = (int)floor(t);
    j = j < 0 ? 0 : (j > kNlna - 2 ? kNlna - 2 : j);
    const double u = t - (double)j, um = 1.0 - u;
    h.j = j;
    h.w0 = (1.0 + 2.0 * u) * um * um;
    h.w1 = u * u * (3.0 - 2.0 * u);
    h.d0 = kDlna * u * um * um;
    h.d1 = kDlna * u * u * (u - 1.0);
    return h;
}

ABCMB_HD Bg10 bg_eval(const double *ot, const HW &h)
{
    Bg10 b;
    const double *r0 = ot + 20 * h.j, *r1 = r0 + 20;
    for (int q = 0; q < B_N; q++)
        b.v[q] = h.w0 * r0[2 * q] + h.w1 * r1[2 * q] + h.d0 * r0[2 * q + 1] + h.d1 * r1[2 * q + 1];
    return b;
}

// d/dln a of the ten interpolated quantities (derivative of the cubic Hermite)
ABCMB_HD Bg10 bg_eval_dlna(const double *ot, double lna)
{
    const double t = (lna - kLna0) * ABCMB_BG_PER_UNIT;
    int j = (int)floor(t);
    j = j < 0 ? 0 : (j > kNlna - 2 ? kNlna - 2 : j);
    const double u = t - (double)j, um = 1.0 - u, s = ABCMB_BG_PER_UNIT;
    const double w0 = -6.0 * u * um * s, w1 = -w0;
    const double d0 = um * (1.0 - 3.0 * u), d1 = u * (3.0 * u - 2.0); // kDlna * s = 1
    Bg10 b;
    const double *r0 = ot + 20 * j, *r1 = r0 + 20;
    for (int q = 0; q < B_N; q++) b.v[q] = w0 * r0[2 * q] + w1 * r1[2 * q] + d0 * r0[2 * q + 1] + d1 * r1[2 * q + 1];
    return b;
}

ABCMB_HD void add_to(double *p, double v)
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    atomicAdd(p, v);
#else
    *p += v;
#endif
}

// adjoint of bg_eval: the table rows' adjoints from the quantities' adjoints
ABCMB_HD void bg_scatter(double *otbar, const HW &h, const Bg10 &bb)
{
    double *r0 = otbar + 20 * h.j, *r1 = r0 + 20;
    for (int q = 0; q < B_N; q++) {
        const double g = bb.v[q];
        if (g == 0.0) continue;
        add_to(r0 + 2 * q, h.w0 * g);
        add_to(r1 + 2 * q, h.w1 * g);
        add_to(r0 + 2 * q + 1, h.d0 * g);
        add_to(r1 + 2 * q + 1, h.d1 * g);
    }
}

// The lanes that share one mode: on the device the 32 lanes of a warp, lane
// i taking the state elements i, i + 32, ...; on the host a single lane, or
// an emulated warp where the host build defines ABCMB_HOST_WARPS (the CPU
// tests).
// Every operator below is called by all lanes of the mode alike, reads its
// inputs, writes only its own lane's elements of the output, and ends with a
// lane barrier, so the next operator may read any element.
ABCMB_HD int ln_id()
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    return threadIdx.x & 31;
#else
    return 0;
#endif
}

ABCMB_HD int ln_n()
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    return 32;
#else
    return 1;
#endif
}

ABCMB_HD void ln_sync()
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    __syncwarp();
#endif
}

ABCMB_HD double ln_sum(double v)
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
    return v;
}

// maximum over the lanes; a NaN anywhere gives NaN
ABCMB_HD double ln_max(double v)
{
#if defined(__CUDA_ARCH__) || defined(ABCMB_HOST_WARPS)
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        if (!(u <= v)) v = u;
    }
#endif
    return v;
}

// streaming coefficients of chain moment l under truncation L
ABCMB_HD void sc_AB(const StreamCoef &sc, int l, int L, double &A, double &Bc)
{
    A = l < L ? sc.a[l] : (l == L ? 1.0 : 0.0);
    Bc = l < L ? sc.b[l] : 0.0;
}

// chain (0 photon temperature, 1 polarization, 2 neutrinos), moment l, its
// truncation L and first element i0 of state element i >= 4
ABCMB_HD void chain_of(const OdeDims &d, int i, int &ch, int &l, int &L, int &i0)
{
    ch = i < d.iG ? 0 : (i < d.iN ? 1 : 2);
    i0 = ch == 0 ? d.iF : (ch == 1 ? d.iG : d.iN);
    L = ch == 0 ? d.Lg : (ch == 1 ? d.Lp : d.Ln);
    l = i - i0;
}

// ---- E: everything but Thomson ----
// hp = 2 kH^2 eta + 3 (fc dc + fb db + fg F0 + fn N0), ep = 1.5 hc / k (fb tb / k + fg F1 + fn N1)
ABCMB_HD void op_E(const OdeDims &d, const StreamCoef &sc, double k, const Bg10 &b, Vec y, Vec out, double fac)
{
    const double ih = b.v[B_IH], kH = k * ih, ik = 1.0 / k;
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    double drho, rpth_k, rpsig;
    ncdm_sums(d, b, y, drho, rpth_k, rpsig);
    const double hp = 2.0 * kH * kH * eta +
                      3.0 * (b.v[B_FC] * dc + b.v[B_FB] * db + b.v[B_FG] * y[d.iF] + b.v[B_FNU] * y[d.iN] + drho);
    const double ep = 1.5 * b.v[B_HC] * ik *
                      (b.v[B_FB] * tb * ik + b.v[B_FG] * y[d.iF + 1] + b.v[B_FNU] * y[d.iN + 1] + rpth_k);
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double f;
        if (i >= d.iM) {
            // massive neutrinos (App. C.6), bin j, moment l
            const int j = (i - d.iM) / (d.Lm + 1), l = i - d.iM - j * (d.Lm + 1), L = d.Lm;
            const double q = ncdm_q(j), eps = sqrt(q * q + b.nx * b.nx);
            const double v = q * k / eps * ih, dlnf = -q / (1.0 + exp(-q));
            if (l == 0) f = -v * y[i + 1] + hp / 6.0 * dlnf;
            else if (l == 1) f = v / 3.0 * (y[i - 1] - 2.0 * y[i + 1]);
            else if (l == 2) f = v / 5.0 * (2.0 * y[i - 1] - 3.0 * y[i + 1]) - (hp / 15.0 + 0.4 * ep) * dlnf;
            else if (l < L) f = v / (2.0 * l + 1.0) * (l * y[i - 1] - (l + 1.0) * y[i + 1]);
            else f = v * y[i - 1] - (L + 1.0) * b.v[B_IHT] * y[i];
        } else if (i < 4) {
            f = i == 0 ? ep : (i == 1 ? -0.5 * hp : (i == 2 ? -ih * tb - 0.5 * hp : -tb + b.v[B_CS2] * k * k * ih * db));
        } else {
            int ch, l, L, i0;
            chain_of(d, i, ch, l, L, i0);
            double A, Bc;
            sc_AB(sc, l, L, A, Bc);
            const double prev = l > 0 ? y[i - 1] : 0.0, nxt = l < L ? y[i + 1] : 0.0;
            f = kH * (A * prev - Bc * nxt);
            if (l == L) f -= (L + 1.0) * b.v[B_IHT] * y[i];
            if (ch != 1 && l == 0) f += -(2.0 / 3.0) * hp;
            if (ch != 1 && l == 2) f += (4.0 / 15.0) * hp + 1.6 * ep;
        }
        out[i] += fac * f;
    }
    ln_sync();
}

ABCMB_HD void op_Et(const OdeDims &d, const StreamCoef &sc, double k, const Bg10 &b, Vec v, Vec out, double fac)
{
    const double ih = b.v[B_IH], kH = k * ih, ik = 1.0 / k;
    const double whp = -0.5 * v[1] - 0.5 * v[2] - (2.0 / 3.0) * (v[d.iF] + v[d.iN]) +
                       (4.0 / 15.0) * (v[d.iF + 2] + v[d.iN + 2]);
    const double wep = v[0] + 1.6 * (v[d.iF + 2] + v[d.iN + 2]);
    const double ce = 1.5 * b.v[B_HC] * ik;
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double g;
        if (i >= d.iM) {
            g = 0.0; // the adjoint covers the massless-neutrino path only
        } else if (i < 4) {
            g = i == 0 ? whp * 2.0 * kH * kH
                       : (i == 1 ? whp * 3.0 * b.v[B_FC]
                                 : (i == 2 ? whp * 3.0 * b.v[B_FB] + v[3] * b.v[B_CS2] * k * k * ih
                                           : wep * ce * b.v[B_FB] * ik - ih * v[2] - v[3]));
        } else {
            // gather form of the transposed streaming: row l receives A_{l+1} v_{l+1} and -B_{l-1} v_{l-1}
            int ch, l, L, i0;
            chain_of(d, i, ch, l, L, i0);
            g = 0.0;
            double A, Bc;
            if (l + 1 <= L) {
                sc_AB(sc, l + 1, L, A, Bc);
                g += kH * A * v[i + 1];
            }
            if (l >= 1) {
                sc_AB(sc, l - 1, L, A, Bc);
                g -= kH * Bc * v[i - 1];
            }
            if (l == L) g -= (L + 1.0) * b.v[B_IHT] * v[i];
            if (ch != 1) {
                const double f = ch == 0 ? b.v[B_FG] : b.v[B_FNU];
                if (l == 0) g += whp * 3.0 * f;
                if (l == 1) g += wep * ce * f;
            }
        }
        out[i] += fac * g;
    }
    ln_sync();
}

ABCMB_HD void op_E_bgrad(const OdeDims &d, const StreamCoef &sc, double k, const Bg10 &b, Vec v, Vec y,
                         double fac, Bg10 &bb)
{
    const double ih = b.v[B_IH], ik = 1.0 / k;
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    const double whp = -0.5 * v[1] - 0.5 * v[2] - (2.0 / 3.0) * (v[d.iF] + v[d.iN]) +
                       (4.0 / 15.0) * (v[d.iF + 2] + v[d.iN + 2]);
    const double wep = v[0] + 1.6 * (v[d.iF + 2] + v[d.iN + 2]);
    const double ce = 1.5 * b.v[B_HC] * ik;
    double stream = 0.0;
    for (int i = 4 + ln_id(); i < d.iM; i += ln_n()) {
        int ch, l, L, i0;
        chain_of(d, i, ch, l, L, i0);
        double A, Bc;
        sc_AB(sc, l, L, A, Bc);
        const double prev = l > 0 ? y[i - 1] : 0.0, nxt = l < L ? y[i + 1] : 0.0;
        stream += v[i] * (A * prev - Bc * nxt);
    }
    stream = ln_sum(stream);
    const double trunc = (d.Lg + 1.0) * v[d.iF + d.Lg] * y[d.iF + d.Lg] +
                         (d.Lp + 1.0) * v[d.iG + d.Lp] * y[d.iG + d.Lp] +
                         (d.Ln + 1.0) * v[d.iN + d.Ln] * y[d.iN + d.Ln];
    bb.v[B_IH] += fac * (whp * 4.0 * k * k * ih * eta + k * stream - v[2] * tb + v[3] * b.v[B_CS2] * k * k * db);
    bb.v[B_IHT] += fac * (-trunc);
    bb.v[B_FC] += fac * whp * 3.0 * dc;
    bb.v[B_FB] += fac * (whp * 3.0 * db + wep * ce * ik * tb);
    bb.v[B_FG] += fac * (whp * 3.0 * y[d.iF] + wep * ce * y[d.iF + 1]);
    bb.v[B_FNU] += fac * (whp * 3.0 * y[d.iN] + wep * ce * y[d.iN + 1]);
    bb.v[B_CS2] += fac * v[3] * k * k * ih * db;
    bb.v[B_HC] += fac * wep * 1.5 * ik * (b.v[B_FB] * tb * ik + b.v[B_FG] * y[d.iF + 1] + b.v[B_FNU] * y[d.iN + 1]);
    ln_sync(); // every lane has read v and y before the caller overwrites them
}

// ---- T: Thomson scattering ----
ABCMB_HD void op_T(const OdeDims &d, double k, const Bg10 &b, Vec y, Vec out, double fac)
{
    const double nu = b.v[B_NU], rnu = b.v[B_RNU];
    const double tb = y[3], F1 = y[d.iF + 1];
    const double Pi = y[d.iF + 2] + y[d.iG] + y[d.iG + 2];
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double g = 0.0;
        if (i == 3) {
            g = rnu * (0.75 * k * F1 - tb);
        } else if (i >= d.iF && i < d.iG) {
            const int l = i - d.iF;
            if (l == 1) g = nu * ((4.0 / 3.0) / k * tb - F1);
            else if (l >= 2) g = -nu * y[i] + (l == 2 ? 0.1 * nu * Pi : 0.0);
        } else if (i >= d.iG && i < d.iN) {
            const int l = i - d.iG;
            g = -nu * y[i] + (l == 0 ? 0.5 * nu * Pi : (l == 2 ? 0.1 * nu * Pi : 0.0));
        }
        out[i] += fac * g;
    }
    ln_sync();
}

ABCMB_HD void op_Tt(const OdeDims &d, double k, const Bg10 &b, Vec v, Vec out, double fac)
{
    const double nu = b.v[B_NU], rnu = b.v[B_RNU];
    const double wpi = 0.1 * v[d.iF + 2] + 0.5 * v[d.iG] + 0.1 * v[d.iG + 2];
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double g = 0.0;
        if (i == 3) {
            g = -rnu * v[3] + nu * (4.0 / 3.0) / k * v[d.iF + 1];
        } else if (i >= d.iF && i < d.iG) {
            const int l = i - d.iF;
            if (l == 1) g = rnu * 0.75 * k * v[3] - nu * v[i];
            else if (l >= 2) g = -nu * v[i] + (l == 2 ? nu * wpi : 0.0);
        } else if (i >= d.iG && i < d.iN) {
            const int l = i - d.iG;
            g = -nu * v[i] + ((l == 0 || l == 2) ? nu * wpi : 0.0);
        }
        out[i] += fac * g;
    }
    ln_sync();
}

ABCMB_HD void op_T_bgrad(const OdeDims &d, double k, Vec v, Vec y, double fac, Bg10 &bb)
{
    const double tb = y[3], F1 = y[d.iF + 1];
    const double Pi = y[d.iF + 2] + y[d.iG] + y[d.iG + 2];
    const double wpi = 0.1 * v[d.iF + 2] + 0.5 * v[d.iG] + 0.1 * v[d.iG + 2];
    double damp = 0.0; // sum of v y over the damped moments (photon l >= 2, all of G)
    for (int i = d.iF + 2 + ln_id(); i < d.iN; i += ln_n()) damp += v[i] * y[i];
    damp = ln_sum(damp);
    const double dnu = v[d.iF + 1] * ((4.0 / 3.0) / k * tb - F1) + wpi * Pi - damp;
    bb.v[B_NU] += fac * dnu;
    bb.v[B_RNU] += fac * v[3] * (0.75 * k * F1 - tb);
    ln_sync(); // every lane has read v and y before the caller overwrites them
}

// y <- (I - h T(b))^{-1} y  (the IMEX implicit part; same algebra as imex_substep)
ABCMB_HD void solve_M(const OdeDims &d, double k, const Bg10 &b, double h, Vec y)
{
    const double hnu = h * b.v[B_NU], hR = h * b.v[B_RNU], dmp = 1.0 / (1.0 + hnu);
    const double rb = y[3], ru = 0.75 * k * y[d.iF + 1];
    const double r2 = y[d.iF + 2], g0 = y[d.iG], g2 = y[d.iG + 2];
    ln_sync(); // every lane has read the coupled elements before any is overwritten
    const double idet = 1.0 / (1.0 + hR + hnu);
    const double pin = (r2 + g0 + g2) / (1.0 + 0.3 * hnu);
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        if (i == 3) y[3] = ((1.0 + hnu) * rb + hR * ru) * idet;
        else if (i == d.iF + 1) y[i] = (hnu * rb + (1.0 + hR) * ru) * idet * (4.0 / 3.0) / k;
        else if (i == d.iF + 2) y[i] = (r2 + 0.1 * hnu * pin) * dmp;
        else if (i == d.iG) y[i] = (g0 + 0.5 * hnu * pin) * dmp;
        else if (i == d.iG + 2) y[i] = (g2 + 0.1 * hnu * pin) * dmp;
        else if ((i >= d.iF + 3 && i < d.iG) || i == d.iG + 1 || (i >= d.iG + 3 && i < d.iN)) y[i] *= dmp;
    }
    ln_sync();
}

// y <- (I - h T(b))^{-T} y
ABCMB_HD void solve_Mt(const OdeDims &d, double k, const Bg10 &b, double h, Vec y)
{
    const double hnu = h * b.v[B_NU], hR = h * b.v[B_RNU], dmp = 1.0 / (1.0 + hnu);
    // (theta_b, F1) block: M2 = [[1 + hR, -hR 3k/4], [-hnu 4/(3k), 1 + hnu]]
    const double a = y[3], c = y[d.iF + 1];
    // (F2, G0, G2): M3 = (1 + hnu) I - hnu c 1^T, c = (0.1, 0.5, 0.1); transpose solve
    const double r2 = y[d.iF + 2], g0 = y[d.iG], g2 = y[d.iG + 2];
    ln_sync();
    const double idet = 1.0 / (1.0 + hR + hnu);
    const double s = (0.1 * r2 + 0.5 * g0 + 0.1 * g2) / (1.0 + 0.3 * hnu);
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        if (i == 3) y[3] = ((1.0 + hnu) * a + hnu * (4.0 / 3.0) / k * c) * idet;
        else if (i == d.iF + 1) y[i] = (hR * 0.75 * k * a + (1.0 + hR) * c) * idet;
        else if (i == d.iF + 2) y[i] = (r2 + hnu * s) * dmp;
        else if (i == d.iG) y[i] = (g0 + hnu * s) * dmp;
        else if (i == d.iG + 2) y[i] = (g2 + hnu * s) * dmp;
        else if ((i >= d.iF + 3 && i < d.iG) || i == d.iG + 1 || (i >= d.iG + 3 && i < d.iN)) y[i] *= dmp;
    }
    ln_sync();
}

// ---- CMB sources at a node (App. B.4 eq. source_functions; see node_sources) ----
// node data: Hc, dHc, g, dg, e^-kappa from the tau-node record
struct NodeD {
    double Hc, dHc, g, dg, emk;
};

ABCMB_HD void sources_fwd(const OdeDims &d, double k, const Bg10 &b, const NodeD &n, const double sw[3], Vec y,
                          double S[3])
{
    const double Hc = n.Hc, k2 = k * k, kH = k / Hc;
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    const double F0 = y[d.iF], F1 = y[d.iF + 1], F2 = y[d.iF + 2], G0 = y[d.iG], G2 = y[d.iG + 2];
    const double N0 = y[d.iN], N1 = y[d.iN + 1], N2 = y[d.iN + 2];
    const double fc = b.v[B_FC], fb = b.v[B_FB], fg = b.v[B_FG], fn = b.v[B_FNU];
    double drho, rpth_k, rpsig;
    ncdm_sums(d, b, y, drho, rpth_k, rpsig);
    const double hp = 2.0 * kH * kH * eta + 3.0 * (fc * dc + fb * db + fg * F0 + fn * N0 + drho);
    const double ep = 1.5 / kH * (fb * tb / k + fg * F1 + fn * N1 + rpth_k);
    const double alpha = Hc * (hp + 6.0 * ep) / (2.0 * k2);
    const double shear = (2.0 / 3.0) * (fg * F2 + fn * N2) + rpsig;
    const double Hap = -2.0 * Hc * alpha + eta - 4.5 * Hc * Hc / k2 * shear;
    const double ap = Hap / Hc;
    const double tbp = -tb + b.v[B_CS2] * k2 * db / Hc + b.v[B_RNU] * (0.75 * k * F1 - tb);
    const double swt = n.g * (0.25 * F0 + Hap);
    const double isw = n.g * (eta - Hap - 2.0 * Hc * alpha) + 2.0 * Hc * n.emk * (ep - n.dHc * alpha - Hap);
    const double dop = Hc * (n.g * (tbp / k2 + ap) + n.dg * (tb / k2 + alpha));
    S[0] = sw[0] * swt + sw[1] * isw + sw[2] * dop;
    S[1] = sw[1] * n.emk * k * (Hap + 2.0 * Hc * alpha - eta);
    S[2] = n.g * (F2 + G0 + G2) * 0.125;
}

// reverse mode of sources_fwd: ybar += dS/dy^T Sbar, bb += dS/db^T Sbar, nb += dS/dn^T Sbar
ABCMB_HD void sources_rev(const OdeDims &d, double k, const Bg10 &b, const NodeD &n, const double sw[3], Vec y,
                          const double Sb[3], Vec yb, Bg10 &bb, NodeD &nb)
{
    const double Hc = n.Hc, k2 = k * k, kH = k / Hc;
    const double eta = y[0], dc = y[1], db = y[2], tb = y[3];
    const double F0 = y[d.iF], F1 = y[d.iF + 1], F2 = y[d.iF + 2];
    const double N0 = y[d.iN], N1 = y[d.iN + 1], N2 = y[d.iN + 2];
    const double fc = b.v[B_FC], fb = b.v[B_FB], fg = b.v[B_FG], fn = b.v[B_FNU];
    const double cs2 = b.v[B_CS2], rnu = b.v[B_RNU];
    // forward intermediates
    const double hp = 2.0 * kH * kH * eta + 3.0 * (fc * dc + fb * db + fg * F0 + fn * N0);
    const double P = fb * tb / k + fg * F1 + fn * N1;
    const double ep = 1.5 / kH * P;
    const double alpha = Hc * (hp + 6.0 * ep) / (2.0 * k2);
    const double shear = (2.0 / 3.0) * (fg * F2 + fn * N2);
    const double Hap = -2.0 * Hc * alpha + eta - 4.5 * Hc * Hc / k2 * shear;
    const double ap = Hap / Hc;
    const double tbp = -tb + cs2 * k2 * db / Hc + rnu * (0.75 * k * F1 - tb);
    const double q1 = Hap + 2.0 * Hc * alpha - eta;
    const double q2 = eta - Hap - 2.0 * Hc * alpha;
    const double q3 = ep - n.dHc * alpha - Hap;
    const double D = n.g * (tbp / k2 + ap) + n.dg * (tb / k2 + alpha);
    // reverse
    const double swtb = sw[0] * Sb[0], iswb = sw[1] * Sb[0], dopb = sw[2] * Sb[0];
    const double q1b = sw[1] * n.emk * k * Sb[1];
    nb.emk += sw[1] * k * q1 * Sb[1];
    // S2
    nb.g += (F2 + y[d.iG] + y[d.iG + 2]) * 0.125 * Sb[2];
    yb[d.iF + 2] += n.g * 0.125 * Sb[2];
    yb[d.iG] += n.g * 0.125 * Sb[2];
    yb[d.iG + 2] += n.g * 0.125 * Sb[2];
    double Hcb = 0.0, Hapb = 0.0, alphab = 0.0, epb = 0.0, hpb = 0.0, etab = 0.0, tbb = 0.0;
    // dop = Hc D
    Hcb += D * dopb;
    const double Db = Hc * dopb;
    nb.g += (tbp / k2 + ap) * Db;
    const double tbpb = n.g / k2 * Db;
    const double apb = n.g * Db;
    nb.dg += (tb / k2 + alpha) * Db;
    tbb += n.dg / k2 * Db;
    alphab += n.dg * Db;
    // isw = g q2 + 2 Hc emk q3
    nb.g += q2 * iswb;
    const double q2b = n.g * iswb;
    Hcb += 2.0 * n.emk * q3 * iswb;
    nb.emk += 2.0 * Hc * q3 * iswb;
    const double q3b = 2.0 * Hc * n.emk * iswb;
    etab += q2b;
    Hapb -= q2b;
    Hcb -= 2.0 * alpha * q2b;
    alphab -= 2.0 * Hc * q2b;
    epb += q3b;
    nb.dHc -= alpha * q3b;
    alphab -= n.dHc * q3b;
    Hapb -= q3b;
    // swt = g (F0 / 4 + Hap)
    nb.g += (0.25 * F0 + Hap) * swtb;
    yb[d.iF] += 0.25 * n.g * swtb;
    Hapb += n.g * swtb;
    // q1 = Hap + 2 Hc alpha - eta
    Hapb += q1b;
    Hcb += 2.0 * alpha * q1b;
    alphab += 2.0 * Hc * q1b;
    etab -= q1b;
    // tbp
    tbb += -tbpb - rnu * tbpb;
    bb.v[B_CS2] += k2 * db / Hc * tbpb;
    yb[2] += cs2 * k2 / Hc * tbpb;
    Hcb -= cs2 * k2 * db / (Hc * Hc) * tbpb;
    bb.v[B_RNU] += (0.75 * k * F1 - tb) * tbpb;
    yb[d.iF + 1] += rnu * 0.75 * k * tbpb;
    // ap = Hap / Hc
    Hapb += apb / Hc;
    Hcb -= Hap / (Hc * Hc) * apb;
    // Hap = -2 Hc alpha + eta - 4.5 Hc^2 / k^2 shear
    Hcb += (-2.0 * alpha - 9.0 * Hc / k2 * shear) * Hapb;
    alphab += -2.0 * Hc * Hapb;
    etab += Hapb;
    const double shearb = -4.5 * Hc * Hc / k2 * Hapb;
    bb.v[B_FG] += (2.0 / 3.0) * F2 * shearb;
    yb[d.iF + 2] += (2.0 / 3.0) * fg * shearb;
    bb.v[B_FNU] += (2.0 / 3.0) * N2 * shearb;
    yb[d.iN + 2] += (2.0 / 3.0) * fn * shearb;
    // alpha = Hc (hp + 6 ep) / (2 k^2)
    Hcb += (hp + 6.0 * ep) / (2.0 * k2) * alphab;
    hpb += Hc / (2.0 * k2) * alphab;
    epb += 6.0 * Hc / (2.0 * k2) * alphab;
    // ep = 1.5 Hc / k P
    Hcb += 1.5 / k * P * epb;
    const double Pb = 1.5 * Hc / k * epb;
    bb.v[B_FB] += tb / k * Pb;
    tbb += fb / k * Pb;
    bb.v[B_FG] += F1 * Pb;
    yb[d.iF + 1] += fg * Pb;
    bb.v[B_FNU] += N1 * Pb;
    yb[d.iN + 1] += fn * Pb;
    // hp = 2 k^2 / Hc^2 eta + 3 (...)
    etab += 2.0 * k2 / (Hc * Hc) * hpb;
    Hcb += -4.0 * k2 * eta / (Hc * Hc * Hc) * hpb;
    bb.v[B_FC] += 3.0 * dc * hpb;
    yb[1] += 3.0 * fc * hpb;
    bb.v[B_FB] += 3.0 * db * hpb;
    yb[2] += 3.0 * fb * hpb;
    bb.v[B_FG] += 3.0 * F0 * hpb;
    yb[d.iF] += 3.0 * fg * hpb;
    bb.v[B_FNU] += 3.0 * N0 * hpb;
    yb[d.iN] += 3.0 * fn * hpb;
    yb[0] += etab;
    yb[3] += tbb;
    nb.Hc += Hcb;
}

// adiabatic initial state (the formulas of initial_state, R_nu given explicitly)
// x0: the massive neutrino's a m / T_ncdm at the start; each momentum bin
// carries the massless neutrinos' adiabatic F_0..F_2 (the species is
// relativistic then): Psi_0 = -F_0 dlnf / 4, Psi_1 = -eps F_1 dlnf / (4 q),
// Psi_2 = -F_2 dlnf / 4
ABCMB_HD void initial_fwd(const OdeDims &d, double k, double tau_i, double Rn, Vec y, double x0 = 0.0)
{
    const double C = 0.5, kt = k * tau_i;
    const double dg = -(2.0 / 3.0) * C * kt * kt;
    const double F1 = -(2.0 / 27.0) * C * kt * kt * kt;
    const double tg = -C * k * kt * kt * kt / 18.0;
    const double N1 = F1 * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn), N2 = (8.0 / 3.0) * C * kt * kt / (15.0 + 4.0 * Rn);
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double v = 0.0;
        if (i >= d.iM) {
            const int j = (i - d.iM) / (d.Lm + 1), l = i - d.iM - j * (d.Lm + 1);
            const double q = ncdm_q(j), eps = sqrt(q * q + x0 * x0), dlnf = -q / (1.0 + exp(-q));
            v = l == 0 ? -0.25 * dg * dlnf : (l == 1 ? -eps / (4.0 * q) * N1 * dlnf : (l == 2 ? -0.25 * N2 * dlnf : 0.0));
            y[i] = v;
            continue;
        }
        if (i == 0) v = 2.0 * C - C * kt * kt * (5.0 + 4.0 * Rn) / (6.0 * (15.0 + 4.0 * Rn));
        else if (i == 1 || i == 2) v = 0.75 * dg;
        else if (i == 3) v = tg;
        else if (i == d.iF || i == d.iN) v = dg;
        else if (i == d.iF + 1) v = F1;
        else if (i == d.iN + 1) v = F1 * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn);
        else if (i == d.iN + 2) v = (8.0 / 3.0) * C * kt * kt / (15.0 + 4.0 * Rn);
        y[i] = v;
    }
    ln_sync();
}

// d/d tau_i of the initial state, dotted with ybar
ABCMB_HD double initial_dtau(const OdeDims &d, double k, double tau_i, double Rn, Vec yb)
{
    const double C = 0.5, kt = k * tau_i, dkt = k;
    const double ddg = -(4.0 / 3.0) * C * kt * dkt;
    const double dF1 = -(6.0 / 27.0) * C * kt * kt * dkt;
    const double dtg = -C * k * 3.0 * kt * kt * dkt / 18.0;
    double s = 0.0;
    s += yb[0] * (-C * 2.0 * kt * dkt * (5.0 + 4.0 * Rn) / (6.0 * (15.0 + 4.0 * Rn)));
    s += yb[1] * 0.75 * ddg + yb[2] * 0.75 * ddg + yb[3] * dtg;
    s += yb[d.iF] * ddg + yb[d.iF + 1] * dF1 + yb[d.iN] * ddg;
    s += yb[d.iN + 1] * dF1 * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn);
    s += yb[d.iN + 2] * (8.0 / 3.0) * C * 2.0 * kt * dkt / (15.0 + 4.0 * Rn);
    return s;
}

// d/d R_nu of the initial state, dotted with ybar
ABCMB_HD double initial_dRn(const OdeDims &d, double k, double tau_i, double Rn, Vec yb)
{
    const double C = 0.5, kt = k * tau_i, q = 15.0 + 4.0 * Rn;
    const double F1 = -(2.0 / 27.0) * C * kt * kt * kt;
    // d/dRn of (5+4Rn)/q = (4 q - 4 (5+4Rn))/q^2 = 40/q^2; of (23+4Rn)/q = -32/q^2; of 1/q = -4/q^2
    double s = yb[0] * (-C * kt * kt / 6.0 * 40.0 / (q * q));
    s += yb[d.iN + 1] * F1 * (-32.0) / (q * q);
    s += yb[d.iN + 2] * (8.0 / 3.0) * C * kt * kt * (-4.0) / (q * q);
    return s;
}

} // namespace adj
} // namespace abcmb
