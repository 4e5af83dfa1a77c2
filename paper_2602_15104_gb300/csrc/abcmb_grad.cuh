// Gradient of C_l with respect to the six cosmological parameters: the
// hand-written discrete adjoint of perturb + project + k-quadrature, then
// the pull-back through the background record.
//
//   abcmb_perturb_taped     forward ODE (one warp per mode, abcmb_adjoint.cuh)
//                           recording each mode's accepted steps and
//                           checkpoints in the caller's workspace
//   abcmb_cl_adjoint        Cbar -> Deltabar, and the adjoints of A_s, n_s
//   abcmb_project_adjoint   Deltabar -> Sbar, and the adjoints of the tau-node
//                           positions and weights and of tau_0
//   abcmb_perturb_adjoint   Sbar -> the adjoint of the background record
//                           (ODE table, conformal-time table at the start,
//                           node data, R_nu), replaying each mode's tape
//   abcmb_record_vjp        grad_j = sum_e recbar_e (rec(p + h_j)_e -
//                           rec(p - h_j)_e) / (2 h_j): the background record's
//                           parameter Jacobian by central differences of
//                           abcmb_background_tables (smooth in the parameters:
//                           fixed-step thermal history, converged bisections)
#pragma once

#include "abcmb_adjoint.cuh"
#include "abcmb_bessel.cuh"

namespace abcmb {
namespace adj {

constexpr long kCkpts = kTapeCap / kSeg + 1;
constexpr int kGradThreads = 64; // two modes (warps) per block

// Workspace of a gradient run.  Without a plan every mode's tape holds
// kTapeCap accepted steps.  With a plan (abcmb_grad_plan: from a first pass
// that counted each mode's accepted steps) mode m's tape holds cap_m steps
// and its checkpoints cap_m / kSeg + 1 states: plan[m] and plan[M + 1 + m]
// are the prefix sums of the tape steps and of the checkpoint states over
// the modes before m (plan[M], plan[2M + 1] the totals); the plan is kept in
// the workspace's last region.
struct GradLayout {
    long M, N;
    size_t work, seg, ckpt, tape, res, plan, total; // byte offsets, total bytes
    long tape_steps, ckpt_states;                    // totals
};

__host__ __device__ inline GradLayout grad_layout(int B, int Nk, const OdeDims &d, long tape_steps = -1,
                                                  long ckpt_states = -1)
{
    GradLayout g;
    g.M = (long)B * Nk;
    g.N = d.N;
    g.tape_steps = tape_steps >= 0 ? tape_steps : (long)kTapeCap * g.M;
    g.ckpt_states = ckpt_states >= 0 ? ckpt_states : kCkpts * g.M;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    g.work = take((size_t)V_COUNT * d.N * g.M * sizeof(double));
    g.seg = take((size_t)(kSeg + 1) * d.N * g.M * sizeof(double));
    g.ckpt = take((size_t)g.ckpt_states * d.N * sizeof(double));
    g.tape = take((size_t)g.tape_steps * 3 * sizeof(double));
    g.res = take((size_t)4 * g.M * sizeof(int));
    g.plan = take(tape_steps >= 0 ? (size_t)(2 * g.M + 2) * sizeof(long long) : 0);
    g.total = off;
    return g;
}

// The tape plan (host) from each mode's accepted steps accepted[b][k]: the
// prefix sums grad_layout's comment describes, in the kernels' mode order
// (k-descending, then cosmology) -> the workspace bytes, 0 if a count is
// negative.
inline size_t make_plan(int B, int Nk, const OdeDims &d, const int *accepted, long long *plan)
{
    const long M = (long)B * Nk;
    long long tape = 0, ck = 0;
    for (long m = 0; m < M; m++) {
        const long kidx = Nk - 1 - m / B, b = m % B;
        const int a = accepted[b * Nk + kidx];
        if (a < 0) return 0;
        plan[m] = tape;
        plan[M + 1 + m] = ck;
        tape += a;
        ck += a / kSeg + 1;
    }
    plan[M] = tape;
    plan[2 * M + 1] = ck;
    return grad_layout(B, Nk, d, tape, ck).total;
}

// each mode's vectors contiguous, so that the lanes of its warp read and
// write consecutive elements
__device__ inline ModeBufs mode_bufs(char *ws, const GradLayout &g, long mi, const long long *plan)
{
    ModeBufs m;
    m.work = (double *)(ws + g.work) + mi * V_COUNT * g.N;
    m.seg = (double *)(ws + g.seg) + mi * (kSeg + 1) * g.N;
    if (plan) {
        m.ckpt = (double *)(ws + g.ckpt) + plan[g.M + 1 + mi] * g.N;
        m.tape = (double *)(ws + g.tape) + 3 * plan[mi];
        m.cap = (long)(plan[mi + 1] - plan[mi]);
    } else {
        m.ckpt = (double *)(ws + g.ckpt) + mi * kCkpts * g.N;
        m.tape = (double *)(ws + g.tape) + (long)kTapeCap * 3 * mi;
        m.cap = kTapeCap;
    }
    m.stride = 1;
    return m;
}

__device__ inline ModeCtx mode_ctx(const OdeDims &d, const StreamCoef &sc, const double *bg, long len, int b,
                                   double k, const double sw[3])
{
    ModeCtx c;
    c.d = d;
    c.sc = sc;
    c.rec = bg + (long)b * len;
    c.tab = c.rec + ABCMB_BG_TABLE;
    c.ot = c.rec + ABCMB_BG_ODETAB;
    c.nodes = c.rec + ABCMB_BG_NODES;
    c.k = k;
    c.sw[0] = sw[0];
    c.sw[1] = sw[1];
    c.sw[2] = sw[2];
    c.n_tau = (int)c.rec[ABCMB_S_NTAU];
    c.ncdm_x1 = c.rec[ABCMB_S_NCDM_X1];
    c.ncdm_pH = c.rec[ABCMB_S_NCDM_PREF] * c.rec[ABCMB_S_H0] * c.rec[ABCMB_S_H0];
    return c;
}

__global__ void __launch_bounds__(kGradThreads)
taped_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg, int Lp,
             int Ln, double rtol, double atol, int max_steps, double s_sw, double s_isw, double s_dop, double *S,
             int *status, char *ws, long tape_steps, long ckpt_states, int record, int *accepted)
{
    ABCMB_CTA_SHARED double sa[129], sb[129];
    for (int l = threadIdx.x; l < 129; l += blockDim.x) {
        sa[l] = (double)l / (2.0 * l + 1.0);
        sb[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    __syncthreads();
    const OdeDims d = ode_dims(Lg, Lp, Ln);
    const GradLayout g = grad_layout(B, Nk, d, tape_steps, ckpt_states);
    const long mi = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; // one warp per mode
    if (mi >= g.M) return;
    const int kidx = Nk - 1 - (int)(mi / B), b = (int)(mi % B);
    const double sw[3] = {s_sw, s_isw, s_dop};
    const ModeCtx c = mode_ctx(d, StreamCoef{sa, sb}, bg, len, b, kv[kidx], sw);
    const long long *plan = tape_steps >= 0 ? (const long long *)(ws + g.plan) : nullptr;
    ModeBufs mb;
    if (record) {
        mb = mode_bufs(ws, g, mi, plan);
    } else { // counting pass: work vectors only
        mb.work = (double *)(ws + g.work) + mi * V_COUNT * g.N;
        mb.seg = mb.ckpt = mb.tape = nullptr;
        mb.stride = 1;
        mb.cap = 0;
    }
    double *Sm = S + ((long)b * Nk + kidx) * (long)c.n_tau * 3;
    int *res = (int *)(ws + g.res) + 4 * mi;
    FwdResult r = {ABCMB_OK, 0, 0, 0};
    if (c.rec[ABCMB_S_STATUS] != 0.0) {
        r.status = ABCMB_E_NONFINITE;
        for (int n = ln_id(); n < 3 * c.n_tau; n += ln_n()) Sm[n] = 0.0;
    } else {
        r = fwd_taped(c, mb, rtol, atol, max_steps, Sm, record != 0);
    }
    if (ln_id() == 0) {
        res[0] = r.status;
        res[1] = r.steps;
        res[2] = r.accepted;
        res[3] = r.emit0;
        status[(long)b * Nk + kidx] = r.status;
        if (accepted) accepted[(long)b * Nk + kidx] = r.accepted;
    }
}

// The forward alone, one warp per mode, working vectors from a workspace of
// V_COUNT x N doubles per mode: the path for a massive neutrino (its three
// momentum-bin hierarchies do not fit the four-lanes kernel's layout).
__global__ void __launch_bounds__(kGradThreads)
plain_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg, int Lp,
             int Ln, int Lm, double rtol, double atol, int max_steps, double s_sw, double s_isw, double s_dop,
             double *S, int *status, int *steps, double *work)
{
    ABCMB_CTA_SHARED double sa[129], sb[129];
    for (int l = threadIdx.x; l < 129; l += blockDim.x) {
        sa[l] = (double)l / (2.0 * l + 1.0);
        sb[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    __syncthreads();
    const OdeDims d = ode_dims(Lg, Lp, Ln, Lm);
    const long M = (long)B * Nk;
    const long mi = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; // one warp per mode
    if (mi >= M) return;
    const int kidx = Nk - 1 - (int)(mi / B), b = (int)(mi % B);
    const double sw[3] = {s_sw, s_isw, s_dop};
    const ModeCtx c = mode_ctx(d, StreamCoef{sa, sb}, bg, len, b, kv[kidx], sw);
    ModeBufs mb;
    mb.work = work + mi * V_COUNT * d.N;
    mb.seg = mb.ckpt = mb.tape = nullptr;
    mb.stride = 1;
    double *Sm = S + ((long)b * Nk + kidx) * (long)c.n_tau * 3;
    FwdResult r = {ABCMB_OK, 0, 0, 0};
    if (c.rec[ABCMB_S_STATUS] != 0.0) {
        r.status = ABCMB_E_NONFINITE;
        for (int n = ln_id(); n < 3 * c.n_tau; n += ln_n()) Sm[n] = 0.0;
    } else {
        r = fwd_taped(c, mb, rtol, atol, max_steps, Sm, false);
    }
    if (ln_id() == 0) {
        status[(long)b * Nk + kidx] = r.status;
        if (steps) {
            steps[2 * ((long)b * Nk + kidx)] = r.steps;
            steps[2 * ((long)b * Nk + kidx) + 1] = 0; // substeps not counted on this path
        }
    }
}

__global__ void __launch_bounds__(kGradThreads)
adjoint_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv, int Lg,
               int Lp, int Ln, double s_sw, double s_isw, double s_dop, const double *__restrict__ Sbar, char *ws,
               double *recbar, long tape_steps, long ckpt_states)
{
    ABCMB_CTA_SHARED double sa[129], sb[129];
    for (int l = threadIdx.x; l < 129; l += blockDim.x) {
        sa[l] = (double)l / (2.0 * l + 1.0);
        sb[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    __syncthreads();
    const OdeDims d = ode_dims(Lg, Lp, Ln);
    const GradLayout g = grad_layout(B, Nk, d, tape_steps, ckpt_states);
    const long mi = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; // one warp per mode
    if (mi >= g.M) return;
    const int kidx = Nk - 1 - (int)(mi / B), b = (int)(mi % B);
    const double sw[3] = {s_sw, s_isw, s_dop};
    const ModeCtx c = mode_ctx(d, StreamCoef{sa, sb}, bg, len, b, kv[kidx], sw);
    const long long *plan = tape_steps >= 0 ? (const long long *)(ws + g.plan) : nullptr;
    const ModeBufs mb = mode_bufs(ws, g, mi, plan);
    const int *res = (const int *)(ws + g.res) + 4 * mi;
    const FwdResult r = {res[0], res[1], res[2], res[3]};
    const double *Sb = Sbar + ((long)b * Nk + kidx) * (long)c.n_tau * 3;
    RowAcc acc;
    acc.j = -1;
    bwd(c, mb, Sinks{recbar + (long)b * len, &acc}, r, Sb);
}

// ---- k-quadrature adjoint: grid (ceil(nl / 256), B) ----
__global__ void __launch_bounds__(256)
cl_adjoint_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ Delta,
                  const double *__restrict__ kv, int lmax, const double *__restrict__ Clbar, double *Deltabar,
                  double *recbar)
{
    extern __shared__ double wk[]; // [Nk] weights, then [Nk] ln(k / k_pivot)
    double *lk = wk + Nk;
    ABCMB_CTA_SHARED double red[2][256];
    const int b = blockIdx.y, nl = lmax - 1;
    const double *rec = bg + (long)b * len;
    const double As = rec[ABCMB_S_AS], ns = rec[ABCMB_S_NS];
    for (int i = threadIdx.x; i < Nk; i += blockDim.x) {
        const double lo = log(kv[i > 0 ? i - 1 : i]), hi = log(kv[i < Nk - 1 ? i + 1 : i]);
        lk[i] = log(kv[i] / kKpivot);
        wk[i] = 4.0 * kPi * 0.5 * (hi - lo) * As * exp((ns - 1.0) * lk[i]);
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    double sAs = 0.0, sNs = 0.0;
    if (q < nl) {
        const double *cb = Clbar + (long)b * 3 * nl;
        const double ctt = cb[q], cte = cb[nl + q], cee = cb[2 * nl + q];
        for (int i = 0; i < Nk; i++) {
            const long o = (((long)b * Nk + i) * nl + q) * 2;
            const double dt = Delta[o], de = Delta[o + 1], w = wk[i];
            Deltabar[o] = w * (2.0 * ctt * dt + cte * de);
            Deltabar[o + 1] = w * (cte * dt + 2.0 * cee * de);
            const double c = w * (ctt * dt * dt + cte * dt * de + cee * de * de);
            sAs += c;
            sNs += c * lk[i];
        }
    }
    red[0][threadIdx.x] = sAs / As;
    red[1][threadIdx.x] = sNs;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(recbar + (long)b * len + ABCMB_S_AS, red[0][0]);
        atomicAdd(recbar + (long)b * len + ABCMB_S_NS, red[1][0]);
    }
}

// ---- projection adjoint: one CTA per (cosmology, k); each thread owns nodes ----
// Per node: G_T = sum_l Dbar_T j_l and its x-derivatives G_T', G_T'', G_T''',
// G_E = sum_l Dbar_E c_E(l) j_l and G_E'; then Sbar and the node adjoints.
__global__ void __launch_bounds__(128)
project_adjoint_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ S,
                       const double *__restrict__ kv, int lmax, double scale_pol,
                       const double *__restrict__ Deltabar, double *Sbar, double *recbar)
{
    extern __shared__ double db[]; // [lmax - 1][2]: Dbar_T, Dbar_E c_E
    ABCMB_CTA_SHARED double red[128];
    const int nl = lmax - 1;
    const int blk = blockIdx.x;
    const int kidx = Nk - 1 - blk / B, b = blk % B;
    const double *rec = bg + (long)b * len;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    const double tau0 = rec[ABCMB_S_TAU0];
    const double *nodes = rec + ABCMB_BG_NODES;
    const double *Sm = S + ((long)b * Nk + kidx) * (long)n_tau * 3;
    double *Sbm = Sbar + ((long)b * Nk + kidx) * (long)n_tau * 3;
    double *rb = recbar + (long)b * len;
    const double kk = kv[kidx];
    const double *Db = Deltabar + ((long)b * Nk + kidx) * (long)nl * 2;
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
        const double l = q + 2.0;
        db[2 * q] = Db[2 * q];
        db[2 * q + 1] = Db[2 * q + 1] * sqrt(3.0 * (l + 2.0) * (l + 1.0) * l * (l - 1.0) / 8.0);
    }
    __syncthreads();
    const double s6 = 2.449489742783178;
    double tau0bar = 0.0;
    for (int i = threadIdx.x; i < n_tau; i += blockDim.x) {
        const double *nd = nodes + 8 * i;
        const double w = nd[N_W];
        const double x = kk * (tau0 - nd[N_TAU]);
        const double u = 1.0 / x;
        const double s0 = Sm[3 * i], s1 = Sm[3 * i + 1], sp = Sm[3 * i + 2];
        // the forward kernel's cutoff and starting values (abcmb_spectra.cuh)
        const bool series = x < 1.0;
        // the series path stops at l = 30 in the forward kernel
        const int lc = series ? min(bessel_cut((float)x, lmax), 30) : bessel_cut((float)x, lmax);
        double jm, jc;
        {
            double j0, j1;
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
            jm = j1;
            jc = 3.0 * u * j1 - j0;
            if (series) {
                const double z = x * x;
                double ss = 1.0;
                for (int n = 7; n >= 1; n--) ss = 1.0 - z / (2.0 * n * (4.0 + 2.0 * n + 1.0)) * ss;
                jc = z / 15.0 * ss;
            }
        }
        double t = series ? x * x / 15.0 : 0.0;
        double gT = 0.0, gT1 = 0.0, gT2 = 0.0, gT3 = 0.0, gE = 0.0, gE1 = 0.0;
        // past lc the forward holds j_l at zero, but still adds the j_{l-1}
        // part of j'_l at l = lc + 1
        const int ltop = min(lc + 1, lmax);
        for (int l = 2; l <= ltop; l++) {
            const double L = (double)l, LL = L * (L + 1.0);
            const double j = jc, j1d = jm - (L + 1.0) * u * jc;
            const double j2d = -2.0 * u * j1d - (1.0 - LL * u * u) * j;
            const double j3d = -(4.0 * x * j2d + (2.0 + x * x - LL) * j1d + 2.0 * x * j) * u * u;
            const double dT = db[2 * (l - 2)], dE = db[2 * (l - 2) + 1];
            gT += dT * j;
            gT1 += dT * j1d;
            gT2 += dT * j2d;
            gT3 += dT * j3d;
            gE += dE * j;
            gE1 += dE * j1d;
            double jn;
            if (series) {
                // x^(l+1) / (2l+3)!! times the series, as the forward kernel
                t *= x / (2.0 * L + 3.0);
                const double z = x * x;
                double ss = 1.0;
                for (int n = 7; n >= 1; n--) ss = 1.0 - z / (2.0 * n * (2.0 * (L + 1.0) + 2.0 * n + 1.0)) * ss;
                jn = t * ss;
            } else {
                jn = fma((2.0 * L + 1.0) * u, jc, -jm);
            }
            jm = jc;
            jc = l + 1 <= lc ? jn : 0.0;
        }
        const double s2 = scale_pol * sp, u2 = u * u;
        Sbm[3 * i] = w * gT;
        Sbm[3 * i + 1] = w * gT1;
        Sbm[3 * i + 2] = w * (scale_pol * 0.5 * (3.0 * gT2 + gT) + s6 * u2 * gE);
        const double wbar = s0 * gT + s1 * gT1 + s2 * 0.5 * (3.0 * gT2 + gT) + s6 * sp * u2 * gE;
        const double xbar = w * (s0 * gT1 + s1 * gT2 + s2 * 0.5 * (3.0 * gT3 + gT1) +
                                 s6 * sp * (u2 * gE1 - 2.0 * u2 * u * gE));
        atomicAdd(rb + ABCMB_BG_NODES + 8 * i + N_W, wbar);
        atomicAdd(rb + ABCMB_BG_NODES + 8 * i + N_TAU, -kk * xbar);
        tau0bar += kk * xbar;
    }
    red[threadIdx.x] = tau0bar;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(rb + ABCMB_S_TAU0, red[0]);
}

// grad[b][j] = sum_e recbar[b][e] (rp[b][j][e] - rm[b][j][e]) / (2 h[b][j]); grid (B, 6)
__global__ void __launch_bounds__(256)
record_vjp_kernel(int B, long len, const double *__restrict__ recbar, const double *__restrict__ rp,
                  const double *__restrict__ rm, const double *__restrict__ h, double *grad)
{
    ABCMB_CTA_SHARED double red[256];
    const int b = blockIdx.x, j = blockIdx.y;
    const double *r = recbar + (long)b * len;
    const double *p = rp + ((long)b * ABCMB_NPARAM + j) * len;
    const double *m = rm + ((long)b * ABCMB_NPARAM + j) * len;
    double s = 0.0;
    for (long e = threadIdx.x; e < len; e += blockDim.x) {
        const double g = r[e];
        if (g != 0.0) s += g * (p[e] - m[e]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int t = blockDim.x / 2; t > 0; t >>= 1) {
        if (threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[(long)b * ABCMB_NPARAM + j] = red[0] / (2.0 * h[(long)b * ABCMB_NPARAM + j]);
}

} // namespace adj
} // namespace abcmb
