// Discrete adjoint of the perturbation step, one warp per (cosmology, k) mode
// (host+device; on the host one lane does everything; the GPU kernels in
// abcmb_grad.cuh call these per mode, the 32 lanes sharing the state vectors'
// elements, see ln_id in abcmb_adjoint_ops.cuh).
//
// Forward (fwd_taped): the extrapolated IMEX / Gragg integrator of
// abcmb_ode.cuh on the ODE-table background, landing on every tau node and
// writing the sources there, which also records each accepted step (start,
// size, column count, regime, landing) and checkpoints the state every kSeg
// accepted steps.  Rejected steps do not change the state, so the accepted
// ones define the discrete map from the initial state to the sources.
//
// Backward (bwd): walks the segments last to first; each segment is replayed
// forward from its checkpoint (the same arithmetic, so the same states), then
// its steps are reversed: at a landing the sources' transposed Jacobian adds
// Sbar to ybar; a step's extrapolated value is the Lagrange combination
// sum_i c_{J,i} Z_i of its column values (Neville's tableau evaluated at
// h = 0), so its transpose sends c_{J,i} ybar back through column i, whose
// substeps are recomputed and reversed one by one (abcmb_adjoint_ops.cuh).
// Every background point met on the way gets the adjoint of its ten
// quantities, scattered into the adjoint of the ODE-table rows; the sources
// add adjoints of the node data; the initial state adds the adjoints of the
// conformal-time table entries at the start and of R_nu, and the start
// itself, a_i(k) = min(a_tc, a_k), moves with a_tc or with the root of
// H(a_k) = k / R_large (App. A.1).  The switch to the explicit regime is
// held fixed (its effect on the sources is of the order of the ODE
// tolerance).
#pragma once

#include "abcmb_adjoint_ops.cuh"

namespace abcmb {
namespace adj {

constexpr int kSeg = 64;        // accepted steps per checkpoint
constexpr int kAK = kKmax;      // extrapolation columns
constexpr int kTapeCap = 65536; // accepted steps a mode may take in a gradient run without a plan

// work vectors of a mode (each N long, strided)
enum {
    V_Y = 0,                   // state
    V_T = 1,                   // Neville tableau [kAK]
    V_ZA = V_T + kAK,          // column scratch
    V_ZB,
    V_ST,                      // states of one column, [2 kAK + 1]
    V_AB = V_ST + 2 * kAK + 1, // rolling adjoints [3]
    V_YB = V_AB + 3,           // ybar
    V_YN,                      // ybar accumulator over columns
    V_WT,                      // scratch
    V_CO,                      // one column's value
    V_COUNT
};

struct ModeBufs {
    double *work; // [V_COUNT][N]
    double *seg;  // [kSeg + 1][N]
    double *ckpt; // [cap / kSeg + 1][N]
    double *tape; // [cap][3]: x, H, J | gbs << 8 | land << 9
    long stride;  // element stride of the vectors (1: each mode's vectors contiguous)
    long cap = kTapeCap; // accepted steps the tape holds
};

ABCMB_HD Vec wv(const ModeBufs &m, const OdeDims &d, int v) { return Vec{m.work + (long)v * d.N * m.stride, m.stride}; }
ABCMB_HD Vec segv(const ModeBufs &m, const OdeDims &d, int s) { return Vec{m.seg + (long)s * d.N * m.stride, m.stride}; }
ABCMB_HD Vec ckv(const ModeBufs &m, const OdeDims &d, int c) { return Vec{m.ckpt + (long)c * d.N * m.stride, m.stride}; }

ABCMB_HD void vcopy(const OdeDims &d, Vec a, Vec b)
{
    for (int i = ln_id(); i < d.N; i += ln_n()) b[i] = a[i];
    ln_sync();
}
ABCMB_HD void vzero(const OdeDims &d, Vec a)
{
    for (int i = ln_id(); i < d.N; i += ln_n()) a[i] = 0.0;
    ln_sync();
}

// Lagrange weight of column i in T_{J,J-1}: IMEX nodes h ~ 1/i, Gragg nodes h^2 ~ 1/i^2
ABCMB_HD double lag_w(int J, int i, bool gbs)
{
    double w = 1.0;
    for (int m = 1; m <= J; m++) {
        if (m == i) continue;
        w *= gbs ? (double)i * i / ((double)i * i - (double)m * m) : (double)i / (double)(i - m);
    }
    return w;
}

struct ModeCtx {
    OdeDims d;
    StreamCoef sc;
    const double *rec, *tab, *ot, *nodes;
    double k, sw[3];
    int n_tau;
    // massive neutrino: m / T_ncdm and PREF H0^2 (0 without one); see bg_at
    double ncdm_x1 = 0.0, ncdm_pH = 0.0;
};

// the ten table quantities at ln a, and the massive neutrino's x = a m / T and
// nn = PREF a^-4 / E^2 = PREF H0^2 / (a^2 H_conf^2) there
ABCMB_HD Bg10 bg_at(const ModeCtx &c, double lna)
{
    Bg10 b = bg_eval(c.ot, hw_at(lna));
    if (c.ncdm_pH > 0.0) {
        const double a = exp(lna), hc = b.v[B_HC];
        b.nx = a * c.ncdm_x1;
        b.nn = c.ncdm_pH / (a * a * hc * hc);
    }
    return b;
}

ABCMB_HD NodeD node_at(const ModeCtx &c, int n)
{
    const double *nd = c.nodes + 8 * n;
    return NodeD{nd[N_HC], nd[N_DHC], nd[N_G], nd[N_DG], nd[N_EXPMK]};
}

// one column of a step: IMEX with j substeps or Gragg with 2j, from y into out
// (with keep, ST[m] = state after m substeps, ST[0] = y)
ABCMB_HD void column(const ModeCtx &c, const ModeBufs &mb, double x, double H, int j, bool gbs, Vec y, Vec out,
                     bool keep)
{
    const OdeDims &d = c.d;
    if (!gbs) {
        const double hs = H / j;
        vcopy(d, y, out);
        if (keep) vcopy(d, y, wv(mb, d, V_ST));
        Bg10 bc = bg_at(c, x);
        for (int m = 0; m < j; m++) {
            const double xm = m == j - 1 ? x + H : x + (m + 1) * hs;
            const Bg10 bn = bg_at(c, xm);
            Vec w = wv(mb, d, V_WT);
            vcopy(d, out, w);
            op_E(d, c.sc, c.k, bc, out, w, hs);
            solve_M(d, c.k, bn, hs, w);
            vcopy(d, w, out);
            if (keep) vcopy(d, out, wv(mb, d, V_ST + m + 1));
            bc = bn;
        }
    } else {
        const int n = 2 * j;
        const double hs = H / n;
        Vec za = wv(mb, d, V_ZA), zb = wv(mb, d, V_ZB);
        vcopy(d, y, za);
        vcopy(d, y, zb);
        {
            const Bg10 b0 = bg_at(c, x);
            op_E(d, c.sc, c.k, b0, za, zb, hs);
            op_T(d, c.k, b0, za, zb, hs);
        }
        if (keep) {
            vcopy(d, za, wv(mb, d, V_ST));
            vcopy(d, zb, wv(mb, d, V_ST + 1));
        }
        // za = z_{m-1}, zb = z_m
        for (int m = 1; m < n; m++) {
            const Bg10 bm = bg_at(c, x + m * hs);
            op_E(d, c.sc, c.k, bm, zb, za, 2.0 * hs);
            op_T(d, c.k, bm, zb, za, 2.0 * hs); // za = z_{m+1}
            if (keep) vcopy(d, za, wv(mb, d, V_ST + m + 1));
            Vec t = za;
            za = zb;
            zb = t;
        }
        vcopy(d, zb, out);
    }
}

// Neville update of the tableau V_T with column j's value raw: afterwards
// V_T[s] = T_{j,s}, s < j (IMEX: nodes h ~ 1/j, Gragg: h^2 ~ 1/j^2)
ABCMB_HD void neville(const OdeDims &d, const ModeBufs &mb, Vec raw, int j, bool gbs)
{
    for (int i = ln_id(); i < d.N; i += ln_n()) {
        double cur = raw[i], prev = wv(mb, d, V_T)[i];
        wv(mb, d, V_T)[i] = cur;
        for (int s = 1; s < j; s++) {
            const double f = gbs ? 1.0 / ((double)j * j / ((double)(j - s) * (j - s)) - 1.0)
                                 : (double)(j - s) / (double)s;
            const double nw = cur + (cur - prev) * f;
            prev = wv(mb, d, V_T + s)[i];
            wv(mb, d, V_T + s)[i] = nw;
            cur = nw;
        }
    }
    ln_sync();
}

// the accepted value T_{J,J-1} of a step with J columns, into out
ABCMB_HD void step_value(const ModeCtx &c, const ModeBufs &mb, double x, double H, int J, bool gbs, Vec y, Vec out)
{
    const OdeDims &d = c.d;
    Vec raw = wv(mb, d, V_CO);
    for (int j = 1; j <= J; j++) {
        column(c, mb, x, H, j, gbs, y, raw, false);
        neville(d, mb, raw, j, gbs);
    }
    vcopy(d, wv(mb, d, V_T + J - 1), out);
}

struct FwdResult {
    int status, steps, accepted, emit0;
};

// the sources at node n from state y, written by lane 0 into S[3 n ..]
ABCMB_HD void emit_sources(const ModeCtx &c, int n, Vec y, double *S)
{
    double s3[3];
    sources_fwd(c.d, c.k, bg_at(c, c.nodes[8 * n + N_LNA]), node_at(c, n), c.sw, y, s3);
    if (ln_id() == 0) {
        S[3 * n] = s3[0];
        S[3 * n + 1] = s3[1];
        S[3 * n + 2] = s3[2];
    }
}

// Forward with the tape (record: false runs the same integration without
// writing the tape and checkpoints, which mb may then leave out).  Error
// control as the four-lanes kernel (group floors, slaved moments excluded
// while h / (H tau_c) > kSlavedHnu in the implicit regime).
ABCMB_HD FwdResult fwd_taped(const ModeCtx &c, const ModeBufs &mb, double rtol, double atol, int max_steps,
                             double *S, bool record = true)
{
    const OdeDims &d = c.d;
    FwdResult r = {ABCMB_OK, 0, 0, 0};
    const Cosmo cz = load_cosmo(c.rec);
    double x = cz.lna_tc;
    {
        const double target = c.k / kRlarge;
        if (hconf(cz, cz.lna_tc) < target) {
            double lo = kLna0, hi = cz.lna_tc;
            if (hconf(cz, lo) < target) x = lo;
            else {
                for (int it = 0; it < 100; it++) {
                    const double mid = 0.5 * (lo + hi);
                    if (mid <= lo || mid >= hi) break;
                    if (hconf(cz, mid) > target) lo = mid; else hi = mid;
                }
                x = 0.5 * (lo + hi);
            }
        }
    }
    double x_ns;
    {
        double lo = cz.lna_sw, hi = -2.0;
        for (int it = 0; it < 60; it++) {
            const double mid = 0.5 * (lo + hi);
            const Herm Hm = herm_at(mid);
            if (herm_val(c.tab, Hm, C_NUT, C_DNUT) > kNuNonStiff) lo = mid; else hi = mid;
        }
        x_ns = hi;
    }
    Vec Y = wv(mb, d, V_Y);
    {
        const Herm Hi = herm_at(x);
        initial_fwd(d, c.k, herm_val(c.tab, Hi, C_TAU, C_DTAU), cz.R_nu, Y, exp(x) * c.ncdm_x1);
    }
    int node = 0;
    double h = 1e-3;
    while (node < c.n_tau) {
        const double xn = c.nodes[8 * node + N_LNA];
        double H = h;
        bool land = false;
        if (x + H >= xn) { H = xn - x; land = true; }
        if (H <= 0.0) {
            if (r.accepted == 0) r.emit0++;
            emit_sources(c, node, Y, S);
            node++;
            continue;
        }
        if (++r.steps > max_steps) { r.status = ABCMB_E_MAX_STEPS; break; }
        if (H < 1e-13 && !land) { r.status = ABCMB_E_NONFINITE; break; }
        const bool gbs = x >= x_ns;
        const Bg10 b0 = bg_at(c, x);
        const bool excl = !gbs && H * b0.v[B_NU] > kSlavedHnu;
        double cm[4] = {0, 0, 0, 0};
        for (int i = ln_id(); i < d.N; i += ln_n()) {
            const int g = i < 3 ? 0 : i == 3 ? 1 : i < d.iN ? 2 : 3;
            cm[g] = fmax(cm[g], fabs(Y[i]));
        }
        for (int g = 0; g < 4; g++) cm[g] = ln_max(cm[g]);
        int jacc = 0;
        double err = 0.0;
        Vec raw = wv(mb, d, V_CO);
        for (int j = 1; j <= kAK; j++) {
            column(c, mb, x, H, j, gbs, Y, raw, false);
            neville(d, mb, raw, j, gbs);
            if (j < 2) continue;
            err = 0.0;
            Vec tj = wv(mb, d, V_T + j - 1), tl = wv(mb, d, V_T + j - 2);
            for (int i = ln_id(); i < d.N; i += ln_n()) {
                const int g = i < 3 ? 0 : i == 3 ? 1 : i < d.iN ? 2 : 3;
                if (excl && i >= d.iF + 2 && i < d.iN) continue;
                const double scl = atol + rtol * fmax(fabs(Y[i]), fmax(ABCMB_CHAIN_FLOOR * cm[g], 1e-290));
                const double e = fabs(tj[i] - tl[i]) / scl;
                if (!(e <= err)) err = e;
            }
            err = ln_max(err);
            if (!(err == err)) break;
            if (err <= 1.0) { jacc = j; break; }
        }
        if (!(err == err) || (jacc == 0 && err > 1e300)) { r.status = ABCMB_E_NONFINITE; break; }
        if (jacc) {
            if (record && r.accepted >= mb.cap) { r.status = ABCMB_E_MAX_STEPS; break; }
            if (record && r.accepted % kSeg == 0) vcopy(d, Y, ckv(mb, d, r.accepted / kSeg));
            if (record && ln_id() == 0) {
                double *tp = mb.tape + 3 * (long)r.accepted;
                tp[0] = x;
                tp[1] = H;
                tp[2] = (double)(jacc | (gbs ? 256 : 0) | (land ? 512 : 0));
            }
            r.accepted++;
            vcopy(d, wv(mb, d, V_T + jacc - 1), Y); // as step_value computes it in the replay
            x = land ? xn : x + H;
            double fac = err > 0.0 ? 0.9 * exp(-log(err) / (gbs ? 2 * jacc - 1 : jacc)) : 4.0;
            if (jacc < kAK - 1) fac *= 1.5;
            fac = fmin(4.0, fmax(0.2, fac));
            const double hn = H * fac;
            h = land ? fmax(h, hn) : hn;
            if (land) {
                emit_sources(c, node, Y, S);
                node++;
            }
        } else {
            h = H * fmin(0.9, fmax(0.1, 0.9 * exp(-log(err) / (gbs ? 2 * kAK - 1 : kAK))));
        }
    }
    if (ln_id() == 0)
        for (int n = node; n < c.n_tau; n++) S[3 * n] = S[3 * n + 1] = S[3 * n + 2] = 0.0;
    ln_sync();
    return r;
}

// Adjoint of the ODE table's two rows j, j + 1 (20 entries each), summed
// locally: consecutive substeps mostly fall in the same table interval, so
// their contributions are added to the record (atomically on the device)
// only when the interval changes.  Added directly, every mode of a cosmology
// would contend for the same few addresses at every substep.
struct RowAcc {
    int j;
    double v[40];
};

// Adjoint sink: the adjoint of the background record (same layout as the
// record) and the row accumulator in front of its ODE table.
struct Sinks {
    double *recbar;
    RowAcc *acc;
};

ABCMB_HD void flush_rows(const Sinks &sk)
{
    if (ln_id() != 0) return;
    RowAcc &a = *sk.acc;
    if (a.j >= 0) {
        double *r = sk.recbar + ABCMB_BG_ODETAB + 20 * (long)a.j;
        for (int e = 0; e < 40; e++)
            if (a.v[e] != 0.0) add_to(r + e, a.v[e]);
    }
    a.j = -1;
}

ABCMB_HD void scatter_bg(const Sinks &sk, double lna, const Bg10 &bb)
{
    if (ln_id() != 0) return; // every lane holds the same bb
    const HW h = hw_at(lna);
    RowAcc &a = *sk.acc;
    if (h.j != a.j) {
        flush_rows(sk);
        a.j = h.j;
        for (int e = 0; e < 40; e++) a.v[e] = 0.0;
    }
    for (int q = 0; q < B_N; q++) {
        const double g = bb.v[q];
        a.v[2 * q] += h.w0 * g;
        a.v[2 * q + 1] += h.d0 * g;
        a.v[20 + 2 * q] += h.w1 * g;
        a.v[21 + 2 * q] += h.d1 * g;
    }
}

ABCMB_HD void zero_bg(Bg10 &b)
{
    for (int q = 0; q < B_N; q++) b.v[q] = 0.0;
}

// ybar <- Phi^T ybar for one accepted step (y = its start state)
ABCMB_HD void step_adjoint(const ModeCtx &c, const ModeBufs &mb, const Sinks &sk, double x, double H, int J,
                           bool gbs, Vec y, Vec yb)
{
    const OdeDims &d = c.d;
    Vec acc = wv(mb, d, V_YN);
    vzero(d, acc);
    for (int i = 1; i <= J; i++) {
        const double w = lag_w(J, i, gbs);
        column(c, mb, x, H, i, gbs, y, wv(mb, d, V_CO), true); // states in ST[0..]
        if (!gbs) {
            const double hs = H / i;
            Vec v = wv(mb, d, V_AB);
            for (int e = ln_id(); e < d.N; e += ln_n()) v[e] = w * yb[e];
            ln_sync();
            for (int m = i; m >= 1; m--) {
                // substep m: z_m = M(bn)^-1 (z_{m-1} + hs E(bc) z_{m-1})
                const double xa = x + (m - 1) * hs;
                const double xb = m == i ? x + H : x + m * hs;
                const Bg10 bc = bg_at(c, xa), bn = bg_at(c, xb);
                Vec zin = wv(mb, d, V_ST + m - 1), zout = wv(mb, d, V_ST + m);
                solve_Mt(d, c.k, bn, hs, v); // v = wbar
                Bg10 bbn, bbc;
                zero_bg(bbn);
                zero_bg(bbc);
                op_T_bgrad(d, c.k, v, zout, hs, bbn);
                op_E_bgrad(d, c.sc, c.k, bc, v, zin, hs, bbc);
                scatter_bg(sk, xb, bbn);
                scatter_bg(sk, xa, bbc);
                Vec t = wv(mb, d, V_AB + 1);
                vcopy(d, v, t);
                op_Et(d, c.sc, c.k, bc, t, v, hs); // v = (I + hs E^T) wbar
            }
            for (int e = ln_id(); e < d.N; e += ln_n()) acc[e] += v[e];
            ln_sync();
        } else {
            const int n = 2 * i;
            const double hs = H / n;
            // rolling adjoints: a2 = zbar_{m+1}, a1 = zbar_m, a0 = zbar_{m-1}
            Vec a2 = wv(mb, d, V_AB), a1 = wv(mb, d, V_AB + 1), a0 = wv(mb, d, V_AB + 2);
            for (int e = ln_id(); e < d.N; e += ln_n()) {
                a2[e] = w * yb[e]; // zbar_n
                a1[e] = 0.0;       // zbar_{n-1}
            }
            ln_sync();
            for (int m = n - 1; m >= 1; m--) {
                // z_{m+1} = z_{m-1} + 2 hs f_m(z_m)
                const Bg10 bm = bg_at(c, x + m * hs);
                Vec zm = wv(mb, d, V_ST + m);
                for (int e = ln_id(); e < d.N; e += ln_n()) a0[e] = a2[e]; // zbar_{m-1} = zbar_{m+1} so far
                ln_sync();
                op_Et(d, c.sc, c.k, bm, a2, a1, 2.0 * hs);
                op_Tt(d, c.k, bm, a2, a1, 2.0 * hs);
                Bg10 bb;
                zero_bg(bb);
                op_E_bgrad(d, c.sc, c.k, bm, a2, zm, 2.0 * hs, bb);
                op_T_bgrad(d, c.k, a2, zm, 2.0 * hs, bb);
                scatter_bg(sk, x + m * hs, bb);
                Vec t = a2;
                a2 = a1;
                a1 = a0;
                a0 = t;
            }
            // a2 = zbar_1, a1 = zbar_0 so far; z_1 = z_0 + hs f_0(z_0)
            const Bg10 b0 = bg_at(c, x);
            Vec z0 = wv(mb, d, V_ST);
            for (int e = ln_id(); e < d.N; e += ln_n()) a1[e] += a2[e];
            ln_sync();
            op_Et(d, c.sc, c.k, b0, a2, a1, hs);
            op_Tt(d, c.k, b0, a2, a1, hs);
            Bg10 bb;
            zero_bg(bb);
            op_E_bgrad(d, c.sc, c.k, b0, a2, z0, hs, bb);
            op_T_bgrad(d, c.k, a2, z0, hs, bb);
            scatter_bg(sk, x, bb);
            for (int e = ln_id(); e < d.N; e += ln_n()) acc[e] += a1[e];
            ln_sync();
        }
    }
    vcopy(d, acc, yb);
}

// sources' adjoint at node n for state y: ybar += ..., the sink gets b and
// node data, and the node's position ln a_n: the state there moves with the
// ODE flow, dy/dln a_n = f(y), and the table quantities with their
// interpolant's slope (the steps landing on the node are otherwise frozen)
ABCMB_HD void sources_adjoint(const ModeCtx &c, const ModeBufs &mb, const Sinks &sk, int n, Vec y,
                              const double *Sb, Vec yb)
{
    const OdeDims &d = c.d;
    const double lna = c.nodes[8 * n + N_LNA];
    const Bg10 b = bg_at(c, lna);
    Bg10 bb;
    zero_bg(bb);
    NodeD nb{0, 0, 0, 0, 0};
    Vec ys = wv(mb, d, V_AB), f = wv(mb, d, V_AB + 1);
    vzero(d, ys);
    // scalar reverse mode, on lane 0 (which alone scatters bb and nb below)
    if (ln_id() == 0) sources_rev(d, c.k, b, node_at(c, n), c.sw, y, Sb + 3 * n, ys, bb, nb);
    ln_sync();
    vzero(d, f);
    op_E(d, c.sc, c.k, b, y, f, 1.0);
    op_T(d, c.k, b, y, f, 1.0);
    double lnab = 0.0;
    for (int e = ln_id(); e < d.N; e += ln_n()) {
        lnab += ys[e] * f[e];
        yb[e] += ys[e];
    }
    ln_sync();
    lnab = ln_sum(lnab);
    if (ln_id() != 0) return;
    const Bg10 db = bg_eval_dlna(c.ot, lna);
    for (int q = 0; q < B_N; q++) lnab += bb.v[q] * db.v[q];
    scatter_bg(sk, lna, bb);
    double *nd = sk.recbar + ABCMB_BG_NODES + 8 * n;
    add_to(nd + N_LNA, lnab);
    add_to(nd + N_HC, nb.Hc);
    add_to(nd + N_DHC, nb.dHc);
    add_to(nd + N_G, nb.g);
    add_to(nd + N_DG, nb.dg);
    add_to(nd + N_EXPMK, nb.emk);
}

// Backward pass for a mode whose forward (fwd_taped) returned fr; Sb [n_tau][3]
ABCMB_HD void bwd(const ModeCtx &c, const ModeBufs &mb, const Sinks &sk, const FwdResult &fr, const double *Sb)
{
    const OdeDims &d = c.d;
    if (fr.status != ABCMB_OK) return;
    Vec yb = wv(mb, d, V_YB);
    vzero(d, yb);
    int node = c.n_tau - 1;
    const int nseg = (fr.accepted + kSeg - 1) / kSeg;
    for (int sgi = nseg - 1; sgi >= 0; sgi--) {
        const int s0 = sgi * kSeg, s1 = s0 + kSeg < fr.accepted ? s0 + kSeg : fr.accepted;
        // replay: seg[s - s0] = state at the start of step s, seg[s1 - s0] = after the last
        vcopy(d, ckv(mb, d, sgi), segv(mb, d, 0));
        for (int s = s0; s < s1; s++) {
            const double *tp = mb.tape + 3 * (long)s;
            const int fl = (int)tp[2];
            step_value(c, mb, tp[0], tp[1], fl & 255, (fl & 256) != 0, segv(mb, d, s - s0), segv(mb, d, s - s0 + 1));
        }
        for (int s = s1 - 1; s >= s0; s--) {
            const double *tp = mb.tape + 3 * (long)s;
            const int fl = (int)tp[2];
            if (fl & 512) {
                sources_adjoint(c, mb, sk, node, segv(mb, d, s - s0 + 1), Sb, yb);
                node--;
            }
            step_adjoint(c, mb, sk, tp[0], tp[1], fl & 255, (fl & 256) != 0, segv(mb, d, s - s0), yb);
        }
    }
    // emissions at the start (the start on a node) use the initial state
    Vec y0 = wv(mb, d, V_Y);
    const Cosmo cz = load_cosmo(c.rec);
    if (fr.accepted > 0) vcopy(d, ckv(mb, d, 0), y0);
    while (node >= 0) {
        sources_adjoint(c, mb, sk, node, y0, Sb, yb);
        node--;
    }
    // initial state: tau_i from the conformal-time table at the start, and R_nu
    const double x0 = fr.accepted > 0 ? mb.tape[0] : c.nodes[N_LNA];
    const Herm Hi = herm_at(x0);
    const double tau_i = herm_val(c.tab, Hi, C_TAU, C_DTAU);
    const double taub = initial_dtau(d, c.k, tau_i, cz.R_nu, yb);
    const double rnub = initial_dRn(d, c.k, tau_i, cz.R_nu, yb);
    // the start itself: moving x0 moves the initial state along dy0/dx0 =
    // (d y0 / d tau_i) / H and starts the flow later, so
    // dL/dx0 = taub / H(x0) - ybar0 . f(x0, y0), f the full right-hand side
    const Bg10 b0 = bg_eval(c.ot, hw_at(x0));
    Vec f0 = wv(mb, d, V_WT);
    vzero(d, f0);
    op_E(d, c.sc, c.k, b0, y0, f0, 1.0);
    op_T(d, c.k, b0, y0, f0, 1.0);
    double yf = 0.0;
    for (int i = ln_id(); i < d.N; i += ln_n()) yf += yb[i] * f0[i];
    yf = ln_sum(yf);
    const double xbar = taub * b0.v[B_IH] - yf;
    flush_rows(sk);
    if (ln_id() != 0) return;
    double *tb = sk.recbar + ABCMB_BG_TABLE;
    add_to(tb + 8 * Hi.j + C_TAU, Hi.h00 * taub);
    add_to(tb + 8 * (Hi.j + 1) + C_TAU, Hi.h01 * taub);
    add_to(tb + 8 * Hi.j + C_DTAU, kDlna * Hi.h10 * taub);
    add_to(tb + 8 * (Hi.j + 1) + C_DTAU, kDlna * Hi.h11 * taub);
    add_to(sk.recbar + ABCMB_S_RNU, rnub);
    // x0 = ln a_tc (a record scalar) or the root of H(x) = k / R_large, whose
    // dependence on H0 and the density parameters follows from H = a H0 sqrt(E2)
    const double target = c.k / kRlarge;
    if (!(hconf(cz, cz.lna_tc) < target)) {
        add_to(sk.recbar + ABCMB_S_LNA_TC, xbar);
    } else if (!(hconf(cz, kLna0) < target)) {
        const double a = exp(x0), ia = 1.0 / a;
        const double r = cz.Om_r * ia * ia * ia * ia, m = cz.Om_m * ia * ia * ia;
        const double e2 = r + m + cz.Om_L;
        const double dlnH_dx = 1.0 + 0.5 * (-4.0 * r - 3.0 * m) / e2;
        // dx0/dp = -(d ln H / dp) / (d ln H / dx)
        const double g = -xbar / dlnH_dx;
        add_to(sk.recbar + ABCMB_S_H0, g / cz.H0);
        add_to(sk.recbar + ABCMB_S_OMG, g * 0.5 * ia * ia * ia * ia / e2);
        add_to(sk.recbar + ABCMB_S_OMNU, g * 0.5 * ia * ia * ia * ia / e2);
        add_to(sk.recbar + ABCMB_S_OMB, g * 0.5 * ia * ia * ia / e2);
        add_to(sk.recbar + ABCMB_S_OMC, g * 0.5 * ia * ia * ia / e2);
        add_to(sk.recbar + ABCMB_S_OML, g * 0.5 / e2);
    }
}

} // namespace adj
} // namespace abcmb
