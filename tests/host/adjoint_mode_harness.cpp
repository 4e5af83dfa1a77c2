// Host build of one mode's taped forward and adjoint (abcmb_adjoint.cuh) for
// the CPU tests: the gradient of <Sbar, S> with respect to every entry of the
// background record, against finite differences of the forward.
#include <vector>

#include "abcmb_adjoint.cuh"

using namespace abcmb;
using namespace abcmb::adj;

namespace {
struct Run {
    OdeDims d;
    double a[129], b[129];
    std::vector<double> work, seg, ckpt, tape;
    ModeCtx c;
    ModeBufs mb;
};

void setup(Run &R, const double *rec, double k, int L)
{
    R.d = ode_dims(L, L, L);
    for (int l = 0; l < 129; l++) {
        R.a[l] = (double)l / (2.0 * l + 1.0);
        R.b[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    R.work.assign((size_t)V_COUNT * R.d.N, 0.0);
    R.seg.assign((size_t)(kSeg + 1) * R.d.N, 0.0);
    R.ckpt.assign((size_t)(kTapeCap / kSeg + 1) * R.d.N, 0.0);
    R.tape.assign((size_t)3 * kTapeCap, 0.0);
    R.c.d = R.d;
    R.c.sc = StreamCoef{R.a, R.b};
    R.c.rec = rec;
    R.c.tab = rec + ABCMB_BG_TABLE;
    R.c.ot = rec + ABCMB_BG_ODETAB;
    R.c.nodes = rec + ABCMB_BG_NODES;
    R.c.k = k;
    R.c.sw[0] = R.c.sw[1] = R.c.sw[2] = 1.0;
    R.c.n_tau = (int)rec[ABCMB_S_NTAU];
    R.mb = ModeBufs{R.work.data(), R.seg.data(), R.ckpt.data(), R.tape.data(), 1, kTapeCap};
}
} // namespace

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }
extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

// sig[0..2]: accepted steps, steps tried, and the sum of the accepted steps'
// column counts and regimes -- equal signatures mean the same discrete map
extern "C" int h_fwd(const double *rec, double k, int L, double rtol, double *S, int *sig)
{
    Run R;
    setup(R, rec, k, L);
    const FwdResult fr = fwd_taped(R.c, R.mb, rtol, 1e-14, 10000000, S);
    long js = 0;
    for (int s = 0; s < fr.accepted && s < kTapeCap; s++) js += (long)R.tape[3 * (size_t)s + 2];
    sig[0] = fr.accepted;
    sig[1] = fr.steps;
    sig[2] = (int)(js % 2147483647L);
    return fr.status;
}

extern "C" int h_grad(const double *rec, double k, int L, double rtol, const double *Sb, double *recbar)
{
    Run R;
    setup(R, rec, k, L);
    std::vector<double> S(3 * (size_t)R.c.n_tau);
    const FwdResult fr = fwd_taped(R.c, R.mb, rtol, 1e-14, 10000000, S.data());
    if (fr.status != ABCMB_OK) return fr.status;
    RowAcc acc;
    acc.j = -1;
    bwd(R.c, R.mb, Sinks{recbar, &acc}, fr, Sb);
    return ABCMB_OK;
}

// one accepted step's value and its adjoint (ybar <- Phi^T ybar, table adjoints into recbar)
extern "C" void h_step(const double *rec, double k, int L, double x, double H, int J, int gbs, const double *y,
                       double *out)
{
    Run R;
    setup(R, rec, k, L);
    std::vector<double> yy(y, y + R.d.N);
    step_value(R.c, R.mb, x, H, J, gbs != 0, Vec{yy.data(), 1}, Vec{out, 1});
}

extern "C" void h_step_adj(const double *rec, double k, int L, double x, double H, int J, int gbs, const double *y,
                           double *yb, double *recbar)
{
    Run R;
    setup(R, rec, k, L);
    std::vector<double> yy(y, y + R.d.N);
    RowAcc acc;
    acc.j = -1;
    const Sinks sk{recbar, &acc};
    step_adjoint(R.c, R.mb, sk, x, H, J, gbs != 0, Vec{yy.data(), 1}, Vec{yb, 1});
    flush_rows(sk);
}
