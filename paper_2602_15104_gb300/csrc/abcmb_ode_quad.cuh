// Perturbation ODEs with four lanes per (cosmology, k) mode -- the path
// abcmb_perturb runs.  Same equations and integrator as abcmb_ode.cuh (which
// documents them: IMEX-Euler / Gragg extrapolation, steps landing on every tau
// node), laid out for the GB300 FP64 pipe, whose issue rate bounds this kernel
// (each SM sub-partition's FP64 unit takes one warp instruction per 64
// cycles, so a warp's time is its count of FP64 instructions):
//
//  * A warp holds 8 modes; lane q = 0..3 of a mode's quad owns the Legendre
//    moments l in [qP, qP+P) of each of the three chains (photon
//    temperature, polarization, neutrinos) in registers.  Streaming couples
//    neighbours only, so a substep exchanges one boundary value per chain
//    per direction (two shuffles).  Each moment is held rescaled, u_l =
//    F_l / s_l with s_0 = 1 and s_l = A_l s_{l-1}, A_l the coefficient of
//    F_{l-1} in F_l' = kH (A_l F_{l-1} - B_l F_{l+1}): then u_l' = kH (u_{l-1}
//    - beta_l u_{l+1}), beta_l = B_l A_{l+1}, and the streaming costs two FMAs
//    per moment instead of a multiply and two FMAs.  The equations' other
//    terms (metric, Thomson, sources, tolerances) carry the s_l factors.
//    Lane 0 also owns l <= 2 of every chain, hence the metric sums, both
//    Thomson blocks and the sources; the four
//    scalars (eta, delta_c, delta_b, theta_b) are kept identical in all four
//    lanes.
//  * The background point (10 interpolated quantities) is split over the
//    quad: lane q evaluates ODE-table columns q, q+4 and 8 + (q & 1), each
//    from the record's cubic of its ln a interval (three FMAs), then the
//    values are broadcast inside the quad.
//  * The accepted state and the step's column values live in shared memory
//    ([vector][element][lane], conflict-free; the scalars take one row, lane
//    q of a quad holding scalar q), the inverse error scales in the last
//    column's slot (the last column's values stay in registers); the working
//    vectors of a column live in registers.  The extrapolation is a weighted
//    sum of the column values (ExtTab).
//  * With eight lanes per mode (LQ = 8, abcmb_options.n_wide) a lane owns P
//    moments with P half as large; everything else is the same.
//  * The error norm is max_i |T_j,j-1 - T_j,j-2|_i / (atol + rtol max(|y_i|,
//    f m_g(i))) with y the state at the step start, f the group floor
//    (abcmb_options.err_floor, default 1e-4) and m_g the largest
//    magnitude of i's group (eta/delta_c/delta_b, theta_b, photons, neutrinos);
//    the inverse scales are formed once per step with the approximate
//    reciprocal (a few ulp of float accuracy, ample for step control).
//  * Control flow is warp-uniform: every lane runs every loop (quads that
//    are done, or already accepted their step, compute and discard), so the
//    full-mask shuffles are always legal.  Masked lanes cost the FP64 pipe as
//    much as active ones on this part, so nothing is lost by this.
#pragma once

#include "abcmb_ode.cuh"

namespace abcmb {

constexpr int kQK = 7; // extrapolation columns (orders up to 7 implicit, 13 explicit)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kQLmax = 63;  // highest hierarchy truncation (4 lanes x 16 moments)

__device__ __forceinline__ double rcp_approx(double x)
{
    double r;
#ifdef __CUDA_ARCH__
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
#else
    r = 1.0 / x; // host builds of this header (the CPU tests)
#endif
    return r;
}

// 1/x for normal positive x: the hardware approximation refined by two
// Newton-Raphson steps r <- r + r (1 - x r), each doubling the correct bits
__device__ __forceinline__ double recip(double x)
{
    double r = rcp_approx(x);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// ODE-table columns, (value, d/dln a) pairs -- written by build_background
enum { O_IH = 0, O_IHT, O_FC, O_FB, O_FG, O_FNU, O_NU, O_RNU, O_CS2, O_HC, O_NCOL };
constexpr int kOStride = 2 * O_NCOL;

struct QBg {
    double ih, iht, fc, fb, fg, fnu, nu, rnu, cs2, hc;
};

// position on the uniform ln a grid: interval j and fraction u of it
struct QPos {
    int j;
    double u;
};

__device__ __forceinline__ QPos qpos(double lna)
{
    // (ln a - ln a_0) per unit spacing; scaling by the power of two is exact,
    // so the single rounding of the fma equals that of the subtraction
    const double t = fma(lna, (double)ABCMB_BG_PER_UNIT, -kLna0 * ABCMB_BG_PER_UNIT);
    int j = (int)t; // t >= 0 on the table (ln a >= -18): truncation is floor
    j = j < 0 ? 0 : (j > kNlna - 2 ? kNlna - 2 : j);
    QPos X;
    X.j = j;
    X.u = t - (double)j;
    return X;
}

// ODE-table quantity c at X: the cubic of its interval from the record's
// polynomial section op (abcmb.h), three FMAs
__device__ __forceinline__ double pcol(const double *op, const QPos &X, int c)
{
    const double *pc = op + 40 * X.j + 4 * c;
    return fma(fma(fma(pc[3], X.u, pc[2]), X.u, pc[1]), X.u, pc[0]);
}

// all ten quantities, interpolated by one lane (used for the sources)
__device__ __forceinline__ QBg obg_all(const double *op, double lna)
{
    const QPos X = qpos(lna);
    QBg b;
    b.ih = pcol(op, X, O_IH);
    b.iht = pcol(op, X, O_IHT);
    b.fc = pcol(op, X, O_FC);
    b.fb = pcol(op, X, O_FB);
    b.fg = pcol(op, X, O_FG);
    b.fnu = pcol(op, X, O_FNU);
    b.nu = pcol(op, X, O_NU);
    b.rnu = pcol(op, X, O_RNU);
    b.cs2 = pcol(op, X, O_CS2);
    b.hc = pcol(op, X, O_HC);
    return b;
}

// split over the lanes of a mode and broadcast: with four lanes, lane q
// interpolates columns q, q + 4 and 8 + (q & 1); with eight, columns q and
// 8 + (q & 1)
template <int LQ = 4>
__device__ __forceinline__ QBg qbg(const double *op, double lna, int q, int qb)
{
    const QPos X = qpos(lna);
    QBg b;
    if (LQ == 8) {
        const double v0 = pcol(op, X, q);
        const double v1 = pcol(op, X, O_CS2 + (q & 1));
        b.ih = __shfl_sync(kFull, v0, qb);
        b.iht = __shfl_sync(kFull, v0, qb + 1);
        b.fc = __shfl_sync(kFull, v0, qb + 2);
        b.fb = __shfl_sync(kFull, v0, qb + 3);
        b.fg = __shfl_sync(kFull, v0, qb + 4);
        b.fnu = __shfl_sync(kFull, v0, qb + 5);
        b.nu = __shfl_sync(kFull, v0, qb + 6);
        b.rnu = __shfl_sync(kFull, v0, qb + 7);
        b.cs2 = __shfl_sync(kFull, v1, qb);
        b.hc = __shfl_sync(kFull, v1, qb + 1);
    } else {
        const double v0 = pcol(op, X, q);
        const double v1 = pcol(op, X, q + 4);
        const double v2 = pcol(op, X, O_CS2 + (q & 1));
        b.ih = __shfl_sync(kFull, v0, qb);
        b.iht = __shfl_sync(kFull, v0, qb + 1);
        b.fc = __shfl_sync(kFull, v0, qb + 2);
        b.fb = __shfl_sync(kFull, v0, qb + 3);
        b.fg = __shfl_sync(kFull, v1, qb);
        b.fnu = __shfl_sync(kFull, v1, qb + 1);
        b.nu = __shfl_sync(kFull, v1, qb + 2);
        b.rnu = __shfl_sync(kFull, v1, qb + 3);
        b.cs2 = __shfl_sync(kFull, v2, qb);
        b.hc = __shfl_sync(kFull, v2, qb + 1);
    }
    return b;
}

// Per-chain streaming coefficients in shared memory.  The hierarchy reads
// F_l' = k_H (A_l F_{l-1} - B_l F_{l+1}) with A_l = l/(2l+1), B_l =
// (l+1)/(2l+1) below the truncation, A_L = 1, B_L = 0 at it (the -(L+1)/(H tau)
// F_L term is added separately).  In the rescaled moments u_l = F_l / s_l
// (s_0 = 1, s_l = A_l s_{l-1} up to L, s_l = 1 above) it reads u_l' = k_H
// (u_{l-1} - beta_l u_{l+1}) with beta_l = B_l A_{l+1} (0 from L on); the
// coupling to u_{l-1} is masked above L, so padding moments stay zero.
struct QCoef {
    const volatile double *S, *Bc; // s_l, beta_l [3][64]; volatile: re-read, not held in registers
    int L[3];
    double L1[3]; // L + 1
};

// s_1 = 1/3 and s_2 = 2/15 for every truncation L >= 4 (A_1 = 1/3, A_2 = 2/5)
constexpr double kS1 = 1.0 / 3.0, kS2 = 2.0 / 15.0;

// the coefficient tables of one kernel's chains, filled once per CTA
__device__ __forceinline__ void fill_coef(double *cS, double *cB, const int Ls[3])
{
    for (int i = threadIdx.x; i < 3 * 64; i += blockDim.x) {
        const int ch = i / 64, l = i % 64, L = Ls[ch];
        auto A = [L](int m) { return m < L ? (double)m / (2.0 * m + 1.0) : 1.0; };
        double sl = 1.0;
        for (int m = 1; m <= l && m <= L; m++) sl *= A(m);
        cS[i] = l <= L ? sl : 1.0;
        cB[i] = l < L ? (l + 1.0) / (2.0 * l + 1.0) * A(l + 1) : 0.0;
    }
}

// 1/n for the substep lengths, tabulated so that no column divides
struct InvTab {
    double inv[2 * kQK + 1];
};

constexpr InvTab make_inv()
{
    InvTab t{};
    for (int n = 1; n <= 2 * kQK; n++) t.inv[n] = 1.0 / n;
    return t;
}

__constant__ InvTab c_inv = make_inv();

// Extrapolation of a step's column values z_1..z_j (z_i from n_i substeps) as
// explicit linear combinations, in place of the Aitken-Neville recursion: the
// value extrapolated to h = 0 through points 1..j is sum_i lam[j][i] z_i (Lagrange weights at 0 in x = h
// for the implicit sequence n_i = i, x = h^2 for the Gragg sequence n_i = 2i),
// and the error estimate, that value minus the one through points 2..j, is
// sum_i mu[j][i] z_i.  A column then costs j + 1 operations per element for
// its error and j for the accepted value, against 2j for Aitken-Neville's
// recursion; the weights are at most a few hundred in size, so rounding
// stays ~1e-13 of the state.
struct ExtTab {
    double lam[2][kQK + 1][kQK + 1], mu[2][kQK + 1][kQK + 1]; // [0: implicit, 1: Gragg][j][i]
};

constexpr double ext_x(int g, int i) { return g ? 1.0 / (4.0 * i * i) : 1.0 / i; }

// Lagrange weight at 0 of point i among points a..b
constexpr double ext_lagrange0(int g, int a, int b, int i)
{
    double w = 1.0;
    for (int k = a; k <= b; k++)
        if (k != i) w *= ext_x(g, k) / (ext_x(g, k) - ext_x(g, i));
    return w;
}

constexpr ExtTab make_ext()
{
    ExtTab t{};
    for (int g = 0; g < 2; g++)
        for (int j = 1; j <= kQK; j++)
            for (int i = 1; i <= j; i++) {
                t.lam[g][j][i] = ext_lagrange0(g, 1, j, i);
                t.mu[g][j][i] = t.lam[g][j][i] - (i >= 2 ? ext_lagrange0(g, 2, j, i) : 0.0);
            }
    return t;
}

__constant__ ExtTab c_ext = make_ext();

// per-mode constants
struct QMode {
    double k, ik, k2, k4, c4ik, c05ik, ik3; // k, 1/k, k^2, k/4, 4/k, 1/(2k), 3/k
};

// metric h', eta' from lane 0's state (result broadcast to the quad)
template <int P>
__device__ __forceinline__ void q_metric(const double (&z)[3][P], const double (&zs)[4], const QBg &b,
                                         const QMode &m, int qb, double &hp, double &ep)
{
    const double kH = m.k * b.ih;
    const double src = fma(b.fc, zs[1], fma(b.fb, zs[2], fma(b.fg, z[0][0], b.fnu * z[2][0])));
    const double h1 = fma(2.0 * kH * kH, zs[0], 3.0 * src);
    // (3/2)(H/k^2) (f_b theta_b + f_g theta_g + f_nu theta_nu), theta = (3k/4) F_1 = (k/4) u_1
    const double e1 = (m.c05ik * b.hc) * fma(b.fb * m.ik3, zs[3], fma(b.fg, z[0][1], b.fnu * z[2][1]));
    hp = __shfl_sync(kFull, h1, qb);
    ep = __shfl_sync(kFull, e1, qb);
}

// value of this lane's moment l == L of a chain (0 where the lane does not hold it)
template <int P>
__device__ __forceinline__ double pick_L(const double (&v)[P], int q, int L)
{
    double r = 0.0;
#pragma unroll
    for (int p = 0; p < P; p++) r = (q * P + p == L) ? v[p] : r;
    return r;
}

template <int P>
__device__ __forceinline__ void put_L(double (&v)[P], int q, int L, double x)
{
#pragma unroll
    for (int p = 0; p < P; p++) v[p] = (q * P + p == L) ? x : v[p];
}

// one linearly implicit Euler substep (see imex_substep), in place
template <int P, int LQ = 4>
__device__ __forceinline__ void q_imex(double (&z)[3][P], double (&zs)[4], const QBg &bc, const QBg &bn,
                                       const QMode &m, double hs, int q, int qb, const QCoef &qc)
{
    double hp, ep;
    q_metric<P>(z, zs, bc, m, qb, hp, ep);
    double lft[3], rgt[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        lft[ch] = __shfl_up_sync(kFull, z[ch][P - 1], 1, LQ);
        rgt[ch] = __shfl_down_sync(kFull, z[ch][0], 1, LQ);
    }
    // scalars, explicit
    {
        const double eta = zs[0], dc = zs[1], db = zs[2], tb = zs[3];
        const double hh = 0.5 * hs * hp;
        zs[0] = fma(hs, ep, eta);
        zs[1] = dc - hh;
        zs[2] = fma(-hs * bc.ih, tb, db) - hh;
        zs[3] = fma(hs, fma(bc.cs2 * m.k2 * bc.ih, db, -tb), tb);
    }
    // streaming, explicit
    const double hkH = hs * m.k * bc.ih, htr = hs * bc.iht;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const volatile double *Bc = qc.Bc + 64 * ch;
        const double curL = pick_L<P>(z[ch], q, qc.L[ch]);
        double prev = q == 0 ? 0.0 : lft[ch];
#pragma unroll
        for (int p = 0; p < P; p++) {
            const int l = q * P + p;
            const double cur = z[ch][p];
            const double nxt = p < P - 1 ? z[ch][p + 1] : rgt[ch];
            z[ch][p] = fma(hkH, fma(-Bc[l], nxt, l <= qc.L[ch] ? prev : 0.0), cur);
            prev = cur;
        }
        // truncation -(L+1)/(H tau) F_L
        put_L<P>(z[ch], q, qc.L[ch], fma(-htr * qc.L1[ch], curL, pick_L<P>(z[ch], q, qc.L[ch])));
    }
    if (q == 0) {
        // metric terms of F_0 and F_2 (the latter divided by s_2 = 2/15)
        const double m0 = hs * (-2.0 / 3.0) * hp, m2 = hs * fma(2.0, hp, 12.0 * ep);
        z[0][0] += m0;
        z[0][2] += m2;
        z[2][0] += m0;
        z[2][2] += m2;
    }
    // implicit Thomson part at x_{m+1}: one division for the three denominators
    const double hnu = hs * bn.nu, hRnu = hs * bn.rnu;
    const double d1 = 1.0 + hnu, d2 = fma(0.3, hnu, 1.0), d3 = d1 + hRnu;
    const double d12 = d1 * d2, r = recip(d12 * d3);
    const double dmp = r * (d2 * d3);
#pragma unroll
    for (int p = 0; p < P; p++) {
        const int l = q * P + p;
        z[0][p] *= (l >= 3) ? dmp : 1.0;
        z[1][p] *= (l == 1 || l >= 3) ? dmp : 1.0;
    }
    if (q == 0) {
        const double idet = r * d12, ipin = r * (d1 * d3);
        const double rb = zs[3], ru = m.k4 * z[0][1]; // theta_gamma
        zs[3] = idet * fma(d1, rb, hRnu * ru);
        z[0][1] = (idet * m.c4ik) * fma(hnu, rb, (1.0 + hRnu) * ru);
        const double r2 = z[0][2], g0 = z[1][0], g2 = z[1][2];
        const double hpin = hnu * (fma(kS2, r2 + g2, g0) * ipin); // h nu Pi / (1 + ...)
        z[0][2] = fma(0.75, hpin, r2) * dmp; // (1/10) hpin / s_2
        z[1][0] = fma(0.5, hpin, g0) * dmp;
        z[1][2] = fma(0.75, hpin, g2) * dmp;
    }
    zs[3] = __shfl_sync(kFull, zs[3], qb);
}

// dst += fac f(src), everything explicit (see rhs_axpy)
template <int P, int LQ = 4>
__device__ __forceinline__ void q_rhs_axpy(const double (&s)[3][P], const double (&ss)[4], double (&d)[3][P],
                                           double (&ds)[4], const QBg &b, const QMode &m, double fac, int q,
                                           int qb, const QCoef &qc)
{
    double hp, ep;
    q_metric<P>(s, ss, b, m, qb, hp, ep);
    double lft[3], rgt[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        lft[ch] = __shfl_up_sync(kFull, s[ch][P - 1], 1, LQ);
        rgt[ch] = __shfl_down_sync(kFull, s[ch][0], 1, LQ);
    }
    const double u1 = __shfl_sync(kFull, s[0][1], qb);                     // F_1 / s_1
    const double Pi = __shfl_sync(kFull, fma(kS2, s[0][2] + s[1][2], s[1][0]), qb); // F_2 + G_0 + G_2
    const double tb = ss[3], fhp = fac * hp;
    ds[0] = fma(fac, ep, ds[0]);
    ds[1] = fma(-0.5, fhp, ds[1]);
    ds[2] = fma(-fac * b.ih, tb, ds[2]) - 0.5 * fhp;
    ds[3] = fma(fac, fma(b.cs2 * m.k2 * b.ih, ss[2], fma(b.rnu, fma(m.k4, u1, -tb), -tb)), ds[3]);
    const double fkH = fac * m.k * b.ih, fnu = fac * b.nu, ftr = fac * b.iht;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const volatile double *Bc = qc.Bc + 64 * ch;
        double prev = q == 0 ? 0.0 : lft[ch];
#pragma unroll
        for (int p = 0; p < P; p++) {
            const int l = q * P + p;
            const double cur = s[ch][p];
            const double nxt = p < P - 1 ? s[ch][p + 1] : rgt[ch];
            double v = fma(fkH, fma(-Bc[l], nxt, l <= qc.L[ch] ? prev : 0.0), d[ch][p]);
            if (ch == 0) v = fma((l >= 1) ? -fnu : 0.0, cur, v);
            if (ch == 1) v = fma(-fnu, cur, v);
            d[ch][p] = v;
            prev = cur;
        }
        const double curL = pick_L<P>(s[ch], q, qc.L[ch]);
        put_L<P>(d[ch], q, qc.L[ch], fma(-ftr * qc.L1[ch], curL, pick_L<P>(d[ch], q, qc.L[ch])));
    }
    if (q == 0) {
        // the F_2 rows divided by s_2 = 2/15; the F_1 row by s_1 = 1/3
        const double fPi = fnu * Pi, m2 = fma(2.0, fhp, 12.0 * fac * ep);
        d[0][0] = fma(-2.0 / 3.0, fhp, d[0][0]);
        d[0][1] = fma(fnu * m.c4ik, tb, d[0][1]);
        d[0][2] += fma(0.75, fPi, m2);
        d[1][0] = fma(0.5, fPi, d[1][0]);
        d[1][2] = fma(0.75, fPi, d[1][2]);
        d[2][0] = fma(-2.0 / 3.0, fhp, d[2][0]);
        d[2][2] += m2;
    }
}

// The state components the sources read: photon F_0..F_2, G_0, G_2,
// neutrino F_0..F_2 (lane 0 of a quad), then the four scalars.
constexpr int kSrcComp = 12;

// Sources at a tau node from the state components v (kSrcComp values, order
// above; moments rescaled, u_l = F_l / s_l).
__device__ __forceinline__ void q_sources_v(const double *op, const double *nd, double k, const double sw[3],
                                            const double (&v)[kSrcComp], double *S)
{
    const QBg b = obg_all(op, nd[N_LNA]);
    const double Hc = nd[N_HC], dHc = nd[N_DHC], g = nd[N_G], dg = nd[N_DG], emk = nd[N_EXPMK];
    const double kH = k / Hc, k2 = k * k;
    const double eta = v[8], dc = v[9], db = v[10], tb = v[11];
    const double Fg0 = v[0], Fg1 = kS1 * v[1], Fg2 = kS2 * v[2];
    const double G0 = v[3], G2 = kS2 * v[4];
    const double Fn0 = v[5], Fn1 = kS1 * v[6], Fn2 = kS2 * v[7];
    const double hp = 2.0 * kH * kH * eta + 3.0 * (b.fc * dc + b.fb * db + b.fg * Fg0 + b.fnu * Fn0);
    const double ep = 1.5 / kH * (b.fb * tb / k + b.fg * Fg1 + b.fnu * Fn1);
    const double alpha = Hc * (hp + 6.0 * ep) / (2.0 * k2);
    const double shear = (2.0 / 3.0) * (b.fg * Fg2 + b.fnu * Fn2);
    const double Hap = -2.0 * Hc * alpha + eta - 4.5 * Hc * Hc / k2 * shear;
    const double ap = Hap / Hc;
    const double tbp = -tb + b.cs2 * k2 * db / Hc + b.rnu * (0.75 * k * Fg1 - tb);
    const double swt = g * (0.25 * Fg0 + Hap);
    const double isw = g * (eta - Hap - 2.0 * Hc * alpha) + 2.0 * Hc * emk * (ep - dHc * alpha - Hap);
    const double dop = Hc * (g * (tbp / k2 + ap) + dg * (tb / k2 + alpha));
    S[0] = sw[0] * swt + sw[1] * isw + sw[2] * dop;
    S[1] = sw[1] * emk * k * (Hap + 2.0 * Hc * alpha - eta);
    S[2] = g * (Fg2 + G0 + G2) * 0.125;
}

// element index (in a lane's state rows) of source component c < 8, held by lane 0
template <int P>
__device__ __forceinline__ int src_elem(int c)
{
    return c < 3 ? c : (c == 3 ? P : (c == 4 ? P + 2 : 2 * P + (c - 5)));
}

// Sources at a tau node from the accepted state in shared memory (lane 0).
template <int P>
__device__ __forceinline__ void q_sources(const double *op, const double *nd, double k, const double sw[3],
                                          const double *Y, const double sc[4], double *S)
{
    double v[kSrcComp];
#pragma unroll
    for (int c = 0; c < 8; c++) v[c] = Y[src_elem<P>(c) * 32];
#pragma unroll
    for (int s = 0; s < 4; s++) v[8 + s] = sc[s];
    q_sources_v(op, nd, k, sw, v, S);
}

// scalar q of four (eta, delta_c, delta_b, theta_b): this lane's share of the scalar row
__device__ __forceinline__ double pick4(const double (&v)[4], int q)
{
    return q == 0 ? v[0] : (q == 1 ? v[1] : (q == 2 ? v[2] : v[3]));
}

// all four scalars from the quad's scalar row (lane qb + s holds scalar s)
__device__ __forceinline__ void load_scalars(double (&v)[4], double mine, int qb)
{
#pragma unroll
    for (int s = 0; s < 4; s++) v[s] = __shfl_sync(kFull, mine, qb + s);
}

// maximum over the LQ lanes of a mode
template <int LQ = 4>
__device__ __forceinline__ double quad_max(double v)
{
#pragma unroll
    for (int o = 1; o < LQ; o <<= 1) {
        const double a = __shfl_xor_sync(kFull, v, o);
        if (!(a <= v)) v = a; // NaN propagates
    }
    return v;
}

// Matter power spectrum (App. B.4, eq. PK) from the scalars sc (eta, delta_c,
// delta_b, theta_b) at ln a = lna: P = (2 pi^2 / k^3) A_s (k/k_pivot)^(n_s-1)
// delta_m^2, delta_m = (rho_c delta_c + rho_b delta_b) / (rho_c + rho_b).
__device__ __forceinline__ double q_matter_pk(const double *op, const double *rec, double lna, double k,
                                              const double sc[4])
{
    const QBg b = obg_all(op, lna);
    const double dm = (b.fc * sc[1] + b.fb * sc[2]) / (b.fc + b.fb);
    const double As = rec[ABCMB_S_AS], ns = rec[ABCMB_S_NS];
    return 2.0 * kPi * kPi / (k * k * k) * As * exp((ns - 1.0) * log(k / kKpivot)) * dm * dm;
}

// density-weighted CDM + baryon contrast at ln a (App. B.4 eq. PK's bracket)
__device__ __forceinline__ double q_delta_m(const double *op, double lna, double dc, double db)
{
    const QBg b = obg_all(op, lna);
    return (b.fc * dc + b.fb * db) / (b.fc + b.fb);
}

// Dense output.  Nodes whose e^-kappa is below kNegligibleWeight (before
// recombination) enter every source through a factor e^-kappa or g = H nu
// e^-kappa no larger than ~1e-12 of its peak, so steps pass them freely and
// their state is interpolated linearly.  Elsewhere a step may pass nodes when
// the cubic Hermite interpolant on (y, f) at both step ends is accurate to
// kInterpFrac * rtol: its error is at most (w H)^4 / 384 of a component for
// solutions varying at rate w, and w is bounded by the streaming frequency
// k / H_conf plus the rate at which the Thomson coupling changes, |nu'| /
// max(nu, 1), plus 2 for the background's own evolution, which caps
// H <= (384 kInterpFrac rtol)^(1/4) / w.  Where the cap is shorter than the
// distance to the next node, the step lands on that node instead.
constexpr double kNegligibleWeight = 1e-14;
constexpr double kInterpFrac = 0.1;

__device__ __forceinline__ double dense_rate(const double *ot, double lna, double nu)
{
    int j = (int)((lna - kLna0) * ABCMB_BG_PER_UNIT);
    j = j < 0 ? 0 : (j > kNlna - 1 ? kNlna - 1 : j);
    return fabs(ot[kOStride * j + 2 * O_NU + 1]) / fmax(nu, 1.0) + 2.0;
}

template <int P>
__device__ __forceinline__ void q_zero(double (&w)[3][P], double (&ws)[4])
{
#pragma unroll
    for (int ch = 0; ch < 3; ch++)
#pragma unroll
        for (int p = 0; p < P; p++) w[ch][p] = 0.0;
#pragma unroll
    for (int s = 0; s < 4; s++) ws[s] = 0.0;
}

// the source components of a register vector (lane 0: moments; every lane
// holds the four scalars) into dst[kSrcComp]
template <int P>
__device__ __forceinline__ void q_store_src(double *dst, const double (&v)[3][P], const double (&vs)[4], int q)
{
    if (q == 0) {
        dst[0] = v[0][0];
        dst[1] = v[0][1];
        dst[2] = v[0][2];
        dst[3] = v[1][0];
        dst[4] = v[1][2];
        dst[5] = v[2][0];
        dst[6] = v[2][1];
        dst[7] = v[2][2];
#pragma unroll
        for (int s = 0; s < 4; s++) dst[8 + s] = vs[s];
    }
}

template <int LQ = 4>
__device__ __forceinline__ void q_copy_src(double *dst, const double *src, int q)
{
    for (int c = q; c < kSrcComp; c += LQ) dst[c] = src[c];
}

// the source components of the accepted state (shared memory, mode base
// column Yq = smw + qb) into dst: with four lanes, lane q copies components q,
// q + 4 and the scalar 8 + q; with eight, lane q copies component q and lanes
// 0..3 the scalars
template <int P, int LQ = 4>
__device__ __forceinline__ void q_store_y1(double *dst, const double *Yq, int q)
{
    if (LQ == 8) {
        dst[q] = Yq[src_elem<P>(q) * 32];
        if (q < 4) dst[8 + q] = Yq[3 * P * 32 + q];
    } else {
        dst[q] = Yq[src_elem<P>(q) * 32];
        dst[q + 4] = Yq[src_elem<P>(q + 4) * 32];
        dst[8 + q] = Yq[3 * P * 32 + q];
    }
}

// interpolated source components at fraction th of the step of length H
template <int P>
__device__ __forceinline__ void q_dense(double (&v)[kSrcComp], const double *dq, const double *Yq, double th,
                                        double H, bool hermite)
{
    const double um = 1.0 - th;
    double a0, a1, b0 = 0.0, b1 = 0.0;
    if (hermite) {
        a0 = fma(th + th, um * um, um * um); // (1 + 2 th)(1 - th)^2
        a1 = 1.0 - a0;
        b0 = H * th * um * um;
        b1 = -H * th * th * um;
    } else {
        a0 = um;
        a1 = th;
    }
#pragma unroll
    for (int c = 0; c < kSrcComp; c++) {
        const double y1 = c < 8 ? Yq[src_elem<P>(c) * 32] : Yq[3 * P * 32 + (c - 8)];
        double r = fma(a0, dq[c], a1 * y1);
        if (hermite) r = fma(b0, dq[kSrcComp + c], fma(b1, dq[2 * kSrcComp + c], r));
        v[c] = r;
    }
}

// Integrate the modes of one warp: LQ = 4 lanes per mode (8 modes per warp)
// or LQ = 8 (4 modes per warp, P half as large: a shorter chain of work per
// substep for the most expensive modes); mi is the mode of this lane's group.
// PK: integrate to ln a = x_out only and write the matter power spectrum
// there into pk_out[b][k] instead of the sources (S unused).  DM: write the
// matter contrast delta_m at every tau node into S[b][k][n_tau] instead of
// the sources (every node by landing or Hermite dense output: the linear
// interpolation that the sources allow where e^-kappa < kNegligibleWeight is
// not used).
template <int P, bool PK = false, bool DM = false, int LQ = 4>
__device__ void quad_modes(long mi, long M, int B, int Nk, const double *__restrict__ bg, long len,
                           const double *__restrict__ kv, const QCoef &qc, double rtol, double atol, int max_steps,
                           const double sw[3], double *S, int *status, int *steps, double *smw, double *dn,
                           double efloor, double x_out = 0.0, double *pk_out = nullptr)
{
    constexpr int E = 3 * P + 1; // chain moments, then one scalar per quad lane
    static_assert(LQ == 4 || (LQ == 8 && P >= 4), "four lanes, or eight with lane 0 holding l <= 2");
    const int lane = threadIdx.x & 31, q = lane & (LQ - 1), qb = lane & ~(LQ - 1);
    const bool valid = mi < M;
    const int kidx = valid ? Nk - 1 - (int)(mi / B) : 0;
    const int b = valid ? (int)(mi % B) : 0;
    const double *rec = bg + (long)b * len;
    const double *tab = rec + ABCMB_BG_TABLE;
    const double *ot = rec + ABCMB_BG_ODETAB;
    const double *op = rec + ABCMB_BG_ODEPOLY((long)rec[ABCMB_S_NTAU]);
    const double *nodes = rec + ABCMB_BG_NODES;
    const int n_tau = PK ? 1 : (int)rec[ABCMB_S_NTAU];
    QMode md;
    md.k = kv[kidx];
    md.ik = 1.0 / md.k;
    md.k2 = md.k * md.k;
    md.k4 = 0.25 * md.k;
    md.c4ik = 4.0 * md.ik;
    md.c05ik = 0.5 * md.ik;
    md.ik3 = 3.0 * md.ik;
    const double k = md.k;
    double *Sm = PK ? nullptr : S + ((long)b * Nk + kidx) * (long)n_tau * (DM ? 1 : 3);
    // shared memory of this lane: element e of vector v at smw[(v E + e) 32 + lane]
    double *sl = smw + lane;
    auto Y = [&](int e) -> double & { return sl[e * 32]; };
    auto T = [&](int s, int e) -> double & { return sl[((1 + s) * E + e) * 32]; };

    int stat = ABCMB_OK, nsteps = 0, nsub = 0, node = 0;
    bool done = !valid;
    if (valid && rec[ABCMB_S_STATUS] != 0.0) { stat = ABCMB_E_NONFINITE; done = true; }
    const Cosmo c = load_cosmo(rec);

    // start: a_i = min(a_tc, a_k), k / H(a_k) = R_large (App. A.1)
    double x = c.lna_tc;
    {
        const double target = k / kRlarge;
        if (hconf(c, c.lna_tc) < target) {
            double lo = kLna0, hi = c.lna_tc;
            if (hconf(c, lo) < target) x = lo;
            else {
                for (int it = 0; it < 100; it++) {
                    const double mid = 0.5 * (lo + hi);
                    if (mid <= lo || mid >= hi) break;
                    if (hconf(c, mid) > target) lo = mid; else hi = mid;
                }
                x = 0.5 * (lo + hi);
            }
        }
    }
    // switch to the explicit (GBS) regime where 1/(H tau_c) falls below kNuNonStiff
    double x_ns;
    {
        double lo = c.lna_sw, hi = -2.0;
        for (int it = 0; it < 60; it++) {
            const double mid = 0.5 * (lo + hi);
            const Herm Hm = herm_at(mid);
            if (herm_val(tab, Hm, C_NUT, C_DNUT) > kNuNonStiff) lo = mid; else hi = mid;
        }
        x_ns = hi;
    }
    // adiabatic initial state (see initial_state)
    double z[3][P], zs[4], w[3][P], ws[4];
    {
        const Herm Hi = herm_at(x);
        const double tau_i = herm_val(tab, Hi, C_TAU, C_DTAU);
        const double C = 0.5, Rn = c.R_nu, kt = k * tau_i;
        const double dg = -(2.0 / 3.0) * C * kt * kt;
        const double F1 = -(2.0 / 27.0) * C * kt * kt * kt;
        const double tg = -C * k * kt * kt * kt / 18.0;
#pragma unroll
        for (int ch = 0; ch < 3; ch++)
#pragma unroll
            for (int p = 0; p < P; p++) z[ch][p] = 0.0;
        if (q == 0) { // rescaled: u_1 = F_1 / s_1 = 3 F_1, u_2 = F_2 / s_2 = (15/2) F_2
            z[0][0] = dg;
            z[0][1] = 3.0 * F1;
            z[2][0] = dg;
            z[2][1] = 3.0 * F1 * (23.0 + 4.0 * Rn) / (15.0 + 4.0 * Rn);
            z[2][2] = 20.0 * C * kt * kt / (15.0 + 4.0 * Rn);
        }
        zs[0] = 2.0 * C - C * kt * kt * (5.0 + 4.0 * Rn) / (6.0 * (15.0 + 4.0 * Rn));
        zs[1] = 0.75 * dg;
        zs[2] = 0.75 * dg;
        zs[3] = tg;
#pragma unroll
        for (int ch = 0; ch < 3; ch++)
#pragma unroll
            for (int p = 0; p < P; p++) Y(ch * P + p) = z[ch][p];
        Y(3 * P) = pick4(zs, q);
    }

    // dense output (see kNegligibleWeight): nodes before n_sig carry source weights
    // below kNegligibleWeight; beyond it a step may pass nodes when the
    // interpolation cap allows.  This quad's interpolation data in dn:
    // y0[kSrcComp] f0[kSrcComp] f1[kSrcComp] (lane 0 the chain moments, the
    // scalars by their owners)
    double *dq = dn + (lane / LQ) * 3 * kSrcComp;
    int n_sig = 0;
    if (!DM) { // delta_m is wanted at every node
        int lo = 0, hi = n_tau - 1; // first node whose e^-kappa reaches the threshold
        if (nodes[8 * hi + N_EXPMK] < kNegligibleWeight) lo = hi;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (nodes[8 * mid + N_EXPMK] >= kNegligibleWeight) hi = mid; else lo = mid + 1;
        }
        n_sig = lo;
    }
    const double x_last = nodes[8 * (n_tau - 1) + N_LNA];
    const double theta_int = pow(384.0 * kInterpFrac * rtol, 0.25);
    bool have_y0 = false, have_f0 = false;

    double h = 1e-3, x0 = x;
    while (__any_sync(kFull, !done)) {
        // this quad's step
        bool stepping = !done;
        double xn = x, H = 0.0;
        bool land = false, emit = false, capped = false;
        int dmode = 0; // 0: none or landing on one node, 1: linear, 2: Hermite dense output
        const QBg bx = qbg<LQ>(op, x, q, qb);
        if (stepping) {
            xn = PK ? x_out : nodes[8 * node + N_LNA];
            H = h;
            if (PK && x + H >= xn) { H = xn - x; land = true; }
            else if (x + H >= xn) {
                if (node < n_sig) {
                    const double xs = nodes[8 * n_sig + N_LNA];
                    if (x + H >= xs) { H = xs - x; capped = true; }
                    dmode = 1;
                } else {
                    const double cap = theta_int * recip(fma(k, bx.ih, dense_rate(ot, x, bx.nu)));
                    if (x + cap < xn) { H = xn - x; land = true; }
                    else {
                        if (cap < H) { H = cap; capped = true; }
                        if (x + H > x_last) { H = x_last - x; capped = true; }
                        dmode = 2;
                    }
                }
            }
            if (H <= 0.0) { emit = true; stepping = false; dmode = 0; }
            else if (++nsteps > max_steps) { stat = ABCMB_E_MAX_STEPS; done = true; stepping = false; }
            else if (H < 1e-13 && !land && !capped) { stat = ABCMB_E_NONFINITE; done = true; stepping = false; }
        }
        const bool gbs = __all_sync(kFull, !stepping || x >= x_ns);
        // inverse error scales from the state at the step start; moments slaved
        // to the tight coupling (photon l >= 2, all of G while H/(H tau_c) >
        // kSlavedHnu in the implicit regime) and padding moments get zero
        const bool excl = !gbs && H * bx.nu > kSlavedHnu;
        // the inverse scales occupy the last tableau column's slot, which is
        // written only by the last column, after its element's scale was read
        {
            // magnitudes and tolerances in the moments F_l = s_l u_l
            double cm2 = 0.0, cm3 = 0.0;
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int l = q * P + p;
                z[0][p] = Y(p);
                z[1][p] = Y(P + p);
                z[2][p] = Y(2 * P + p);
                cm2 = fmax(cm2, fmax(fabs(z[0][p]) * qc.S[l], fabs(z[1][p]) * qc.S[64 + l]));
                cm3 = fmax(cm3, fabs(z[2][p]) * qc.S[128 + l]);
            }
            load_scalars(zs, Y(3 * P), qb);
            // floors clamped away from zero keep every scale a normal number
            const double fl0 = fmax(efloor * fmax(fabs(zs[0]), fmax(fabs(zs[1]), fabs(zs[2]))), 1e-290);
            const double fl1 = fmax(efloor * fabs(zs[3]), 1e-290);
            const double fl2 = fmax(efloor * quad_max<LQ>(cm2), 1e-290);
            const double fl3 = fmax(efloor * quad_max<LQ>(cm3), 1e-290);
            // (with eight lanes, lanes 4..7 hold no scalar)
            T(kQK - 1, 3 * P) = q < 4 ? rcp_approx(fma(rtol, fmax(fabs(pick4(zs, q)), q < 3 ? fl0 : fl1), atol)) : 0.0;
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
#pragma unroll
                for (int p = 0; p < P; p++) {
                    const int l = q * P + p;
                    const bool off = l > qc.L[ch] || (excl && (ch == 1 || (ch == 0 && l >= 2)));
                    const double sl = qc.S[64 * ch + l];
                    const double sc = fma(rtol, fmax(fabs(z[ch][p]) * sl, ch < 2 ? fl2 : fl3), atol);
                    T(kQK - 1, ch * P + p) = off ? 0.0 : sl * rcp_approx(sc);
                }
        }
        // interpolation data at the step start (z, zs hold the state here)
        {
            const bool need_f = stepping && dmode == 2 && !have_f0;
            if (__any_sync(kFull, need_f)) {
                q_zero<P>(w, ws);
                q_rhs_axpy<P, LQ>(z, zs, w, ws, bx, md, 1.0, q, qb, qc);
                if (need_f) {
                    q_store_src<P>(dq + kSrcComp, w, ws, q);
                    nsub++;
                }
            }
            if (stepping && dmode >= 1 && !have_y0) q_store_src<P>(dq, z, zs, q);
            have_y0 |= stepping && dmode >= 1;
            have_f0 |= need_f;
        }
        int jacc = 0;
        double err = 0.0;
        bool open = stepping; // still extrapolating this step
        for (int j = 1; j <= kQK; j++) {
            if (!__any_sync(kFull, open)) break;
            if (j > 1) {
                // working vector z := Y (already loaded for j = 1)
#pragma unroll
                for (int ch = 0; ch < 3; ch++)
#pragma unroll
                    for (int p = 0; p < P; p++) z[ch][p] = Y(ch * P + p);
                load_scalars(zs, Y(3 * P), qb);
            }
            if (!gbs) {
                const double hs = H * c_inv.inv[j];
                QBg bc = qbg<LQ>(op, x, q, qb);
                for (int m = 0; m < j; m++) {
                    const double xm = m == j - 1 ? x + H : x + (m + 1) * hs;
                    const QBg bn = qbg<LQ>(op, xm, q, qb);
                    q_imex<P, LQ>(z, zs, bc, bn, md, hs, q, qb, qc);
                    bc = bn;
                }
                if (open) nsub += j;
            } else {
                const int n = 2 * j;
                const double hs = H * c_inv.inv[n];
#pragma unroll
                for (int ch = 0; ch < 3; ch++)
#pragma unroll
                    for (int p = 0; p < P; p++) w[ch][p] = z[ch][p];
#pragma unroll
                for (int s = 0; s < 4; s++) ws[s] = zs[s];
                q_rhs_axpy<P, LQ>(z, zs, w, ws, qbg<LQ>(op, x, q, qb), md, hs, q, qb, qc); // w = z1
                for (int m = 1; m < n; m += 2) {
                    const QBg bm = qbg<LQ>(op, x + m * hs, q, qb);
                    q_rhs_axpy<P, LQ>(w, ws, z, zs, bm, md, 2.0 * hs, q, qb, qc); // z = z_{m+1}
                    if (m + 1 < n) {
                        const QBg bm1 = qbg<LQ>(op, x + (m + 1) * hs, q, qb);
                        q_rhs_axpy<P, LQ>(z, zs, w, ws, bm1, md, 2.0 * hs, q, qb, qc);
                    }
                }
                if (open) nsub += n;
            }
            // column j's value is the j-th point of the extrapolation: kept in
            // slot j - 1 (the last slot holds the inverse error scales, and
            // the last column's value stays in registers); error estimate
            // sum_i mu[j][i] z_i (see ExtTab)
            const double *mw = c_ext.mu[gbs ? 1 : 0][j];
            // max of the scaled errors on the high words of their bit patterns:
            // integer work, monotone for non-negative doubles, NaN on top, exact to 2^-20
            int elh = 0;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int ch = e < 3 * P ? e / P : 3;
                const int p = e - ch * P;
                const double cur = ch < 3 ? z[ch][p] : pick4(zs, q);
                if (j >= 2) {
                    double d = mw[j] * cur;
#pragma unroll
                    for (int i = 1; i < kQK; i++)
                        if (i < j) d = fma(mw[i], T(i - 1, e), d);
                    const double er = fabs(d) * T(kQK - 1, e);
                    elh = max(elh, __double2hiint(er));
                }
                if (j < kQK) T(j - 1, e) = cur;
            }
#pragma unroll
            for (int o = 1; o < LQ; o <<= 1) elh = max(elh, __shfl_xor_sync(kFull, elh, o));
            const double el = __hiloint2double(elh, 0);
            if (open && j >= 2) {
                err = el;
                if (!(el == el)) {
                    stat = ABCMB_E_NONFINITE;
                    done = true;
                    open = false;
                    jacc = -1;
                } else if (el <= 1.0) {
                    jacc = j;
                    open = false;
                    // accepted value sum_i lam[j][i] z_i, z_j from registers
                    const double *lw = c_ext.lam[gbs ? 1 : 0][j];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const int ch = e < 3 * P ? e / P : 3;
                        const int p = e - ch * P;
                        double v = lw[j] * (ch < 3 ? z[ch][p] : pick4(zs, q));
#pragma unroll
                        for (int i = 1; i < kQK; i++)
                            if (i < j) v = fma(lw[i], T(i - 1, e), v);
                        Y(e) = v;
                    }
                }
            }
        }
        if (stepping && jacc == 0 && err > 1e300) {
            stat = ABCMB_E_NONFINITE;
            done = true;
            jacc = -1;
        }
        if (stepping && jacc > 0) {
            x0 = x;
            x = land ? xn : x + H;
            const int ord = gbs ? 2 * jacc - 1 : jacc;
            double fac = err > 0.0 ? 0.9 * (double)__powf((float)err, -1.0f / ord) : 4.0;
            if (jacc < kQK - 1) fac *= 1.5;
            fac = fmin(4.0, fmax(0.2, fac));
            const double hn = H * fac;
            h = (land || capped) ? fmax(h, hn) : hn;
            if (land) emit = true;
        } else if (stepping && jacc == 0) {
            const int ord = gbs ? 2 * kQK - 1 : kQK;
            h = H * fmin(0.9, fmax(0.1, 0.9 * (double)__powf((float)err, -1.0f / ord)));
        }
        // dense output of the nodes in (x0, x]
        bool pend = stepping && jacc > 0 && dmode >= 1;
        if (__any_sync(kFull, pend && dmode == 2)) {
            // f1 at the step end
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
#pragma unroll
                for (int p = 0; p < P; p++) z[ch][p] = Y(ch * P + p);
            load_scalars(zs, Y(3 * P), qb);
            q_zero<P>(w, ws);
            q_rhs_axpy<P, LQ>(z, zs, w, ws, qbg<LQ>(op, x, q, qb), md, 1.0, q, qb, qc);
            if (pend && dmode == 2) {
                q_store_src<P>(dq + 2 * kSrcComp, w, ws, q);
                nsub++;
            }
        }
        if (__any_sync(kFull, pend)) {
            __syncwarp();
            const double iH = pend ? recip(x - x0) : 0.0;
            while (__any_sync(kFull, pend)) {
                const int i = node + q;
                const bool mine = pend && i < n_tau && nodes[8 * i + N_LNA] <= x;
                if (mine) {
                    const double th = fmin((nodes[8 * i + N_LNA] - x0) * iH, 1.0);
                    double v[kSrcComp];
                    q_dense<P>(v, dq, smw + qb, th, x - x0, dmode == 2);
                    if (DM) Sm[i] = q_delta_m(op, nodes[8 * i + N_LNA], v[9], v[10]);
                    else q_sources_v(op, nodes + 8 * i, k, sw, v, Sm + 3 * i);
                }
                const int cnt = __popc((__ballot_sync(kFull, mine) >> qb) & ((1u << LQ) - 1u));
                if (pend) {
                    node += cnt;
                    if (node >= n_tau) done = true;
                    if (cnt < LQ || done) pend = false;
                }
            }
            __syncwarp();
        }
        if (stepping && jacc > 0) {
            // the step end is the next step's start
            if (dmode >= 1) {
                if (dmode == 2) q_copy_src<LQ>(dq + kSrcComp, dq + 2 * kSrcComp, q);
                q_store_y1<P, LQ>(dq, smw + qb, q);
            }
            have_y0 = dmode >= 1;
            have_f0 = dmode == 2;
        }
        __syncwarp();
        if (__any_sync(kFull, emit)) {
            double sc[4];
            load_scalars(sc, Y(3 * P), qb); // the accepted scalars, one per quad lane
            if (emit) {
                if (q == 0) {
                    if (PK) pk_out[(long)b * Nk + kidx] = q_matter_pk(op, rec, x_out, k, sc);
                    else if (DM) Sm[node] = q_delta_m(op, nodes[8 * node + N_LNA], sc[1], sc[2]);
                    else q_sources<P>(op, nodes + 8 * node, k, sw, sl, sc, Sm + 3 * node);
                }
                node++;
                if (node >= n_tau) done = true;
            }
        }
    }
    if (valid && q == 0) {
        if (PK) {
            if (node < 1) pk_out[(long)b * Nk + kidx] = nan("");
        } else if (DM) {
            for (int n = node; n < n_tau; n++) Sm[n] = 0.0;
        } else {
            for (int n = node; n < n_tau; n++) Sm[3 * n] = Sm[3 * n + 1] = Sm[3 * n + 2] = 0.0;
        }
        status[(long)b * Nk + kidx] = stat;
        if (steps) {
            steps[2 * ((long)b * Nk + kidx)] = nsteps;
            steps[2 * ((long)b * Nk + kidx) + 1] = nsub;
        }
    }
}

// Dynamic shared memory of one warp: the accepted state and the K tableau
// columns, (1 + K) (3P + 1) doubles per lane, then the 8 quads' dense-output
// data, 3 kSrcComp doubles each.
template <int P>
constexpr size_t quad_smem_per_warp()
{
    return ((size_t)(1 + kQK) * (3 * P + 1) * 32 + 8 * 3 * kSrcComp) * sizeof(double);
}

// Modes (k-descending, then cosmology) [0, M8) run eight lanes each in the
// first nb8 one-warp CTAs (the highest k: their per-substep chain of work is
// what bounds the launch); the rest run four lanes each.  W = 1 whenever
// nb8 > 0.  Both layouts evaluate the same expressions for a mode; its warp-
// mates differ, which moves the warp-wide switch to the explicit regime.
template <int P, int W>
__global__ void __launch_bounds__(32 * W)
perturb_quad_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg,
                    int Lp, int Ln, double rtol, double atol, int max_steps, double s_sw, double s_isw,
                    double s_dop, double *S, int *status, int *steps, int nb8, long M8, double efloor)
{
    extern __shared__ double qsm[];
    ABCMB_CTA_SHARED double cS[3 * 64], cB[3 * 64];
    const int Ls[3] = {Lg, Lp, Ln};
    fill_coef(cS, cB, Ls);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long M = (long)B * Nk;
    QCoef qc;
    qc.S = cS;
    qc.Bc = cB;
    qc.L[0] = Lg;
    qc.L[1] = Lp;
    qc.L[2] = Ln;
    for (int c = 0; c < 3; c++) qc.L1[c] = qc.L[c] + 1.0;
    const double sw[3] = {s_sw, s_isw, s_dop};
    if constexpr (P >= 8) {
        if ((int)blockIdx.x < nb8) {
            constexpr int P8 = P / 2, E8 = 3 * P8 + 1;
            const long mi = (long)blockIdx.x * 4 + (lane >> 3);
            quad_modes<P8, false, false, 8>(mi, M8, B, Nk, bg, len, kv, qc, rtol, atol, max_steps, sw, S, status,
                                            steps, qsm, qsm + (1 + kQK) * E8 * 32, efloor);
            return;
        }
    }
    constexpr int E = 3 * P + 1;
    const long mi = M8 + ((long)(blockIdx.x - nb8) * W + warp) * 8 + (lane >> 2);
    double *smw = qsm + (long)warp * ((1 + kQK) * E * 32 + 8 * 3 * kSrcComp);
    quad_modes<P>(mi, M, B, Nk, bg, len, kv, qc, rtol, atol, max_steps, sw, S, status, steps, smw,
                  smw + (1 + kQK) * E * 32, efloor);
}

// Matter power spectrum at ln a = x_out for every (cosmology, k) mode: the
// perturbation ODE alone, with no tau nodes to land on.
template <int P>
__global__ void __launch_bounds__(32)
pk_quad_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg,
               int Lp, int Ln, double rtol, double atol, int max_steps, double x_out, double *Pk, int *status,
               int *steps, double efloor)
{
    extern __shared__ double qsm[];
    ABCMB_CTA_SHARED double cS[3 * 64], cB[3 * 64];
    const int Ls[3] = {Lg, Lp, Ln};
    fill_coef(cS, cB, Ls);
    __syncthreads();
    constexpr int E = 3 * P + 1;
    const int lane = threadIdx.x & 31;
    const long M = (long)B * Nk;
    const long mi = (long)blockIdx.x * 8 + (lane >> 2);
    QCoef qc;
    qc.S = cS;
    qc.Bc = cB;
    qc.L[0] = Lg;
    qc.L[1] = Lp;
    qc.L[2] = Ln;
    for (int c = 0; c < 3; c++) qc.L1[c] = qc.L[c] + 1.0;
    const double sw[3] = {0.0, 0.0, 0.0};
    quad_modes<P, true>(mi, M, B, Nk, bg, len, kv, qc, rtol, atol, max_steps, sw, nullptr, status, steps, qsm,
                        qsm + (1 + kQK) * E * 32, efloor, x_out, Pk);
}

// delta_m at every tau node for every (cosmology, k) mode: Dm[B][Nk][n_tau]
template <int P>
__global__ void __launch_bounds__(32)
dm_quad_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg,
               int Lp, int Ln, double rtol, double atol, int max_steps, double *Dm, int *status, double efloor)
{
    extern __shared__ double qsm[];
    ABCMB_CTA_SHARED double cS[3 * 64], cB[3 * 64];
    const int Ls[3] = {Lg, Lp, Ln};
    fill_coef(cS, cB, Ls);
    __syncthreads();
    constexpr int E = 3 * P + 1;
    const int lane = threadIdx.x & 31;
    const long M = (long)B * Nk;
    const long mi = (long)blockIdx.x * 8 + (lane >> 2);
    QCoef qc;
    qc.S = cS;
    qc.Bc = cB;
    qc.L[0] = Lg;
    qc.L[1] = Lp;
    qc.L[2] = Ln;
    for (int c = 0; c < 3; c++) qc.L1[c] = qc.L[c] + 1.0;
    const double sw[3] = {1.0, 1.0, 1.0};
    quad_modes<P, false, true>(mi, M, B, Nk, bg, len, kv, qc, rtol, atol, max_steps, sw, Dm, status, nullptr,
                               qsm, qsm + (1 + kQK) * E * 32, efloor);
}

} // namespace abcmb
