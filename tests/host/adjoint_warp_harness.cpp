// Host build of one mode's taped forward and adjoint (abcmb_adjoint.cuh) on
// an emulated warp for the CPU tests: the 32 lanes share the mode's state
// elements as taped_kernel and adjoint_kernel run them (lane sums, maxima,
// barriers and the record adjoint's atomic additions through warp_emu.h).
#define ABCMB_HOST_WARPS
#include "warp_emu.h"

#include <vector>

#include "abcmb_adjoint.cuh"

using namespace abcmb;
using namespace abcmb::adj;

namespace {
// the mode's context and buffers, shared by its lanes as device memory is
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

FwdResult forward(Run &R, double rtol, double *S)
{
    FwdResult fr{};
    emu::run_cta(0, 0, 32, [&] {
        const FwdResult r = fwd_taped(R.c, R.mb, rtol, 1e-14, 10000000, S);
        if (threadIdx.x == 0) fr = r;
    });
    return fr;
}
} // namespace

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

// sources S[n_tau][3] of one mode at L; sig as the one-lane harness's h_fwd
// (accepted steps, steps tried, sum of the accepted steps' column counts and regimes)
extern "C" int h_fwd_warp(const double *rec, double k, int L, double rtol, double *S, int *sig)
{
    Run R;
    setup(R, rec, k, L);
    const FwdResult fr = forward(R, rtol, S);
    long js = 0;
    for (int s = 0; s < fr.accepted && s < kTapeCap; s++) js += (long)R.tape[3 * (size_t)s + 2];
    sig[0] = fr.accepted;
    sig[1] = fr.steps;
    sig[2] = (int)(js % 2147483647L);
    return fr.status;
}

// recbar += d<Sb, S>/d(record), the taped forward then the reverse sweep
extern "C" int h_grad_warp(const double *rec, double k, int L, double rtol, const double *Sb, double *recbar)
{
    Run R;
    setup(R, rec, k, L);
    std::vector<double> S(3 * (size_t)R.c.n_tau);
    const FwdResult fr = forward(R, rtol, S.data());
    if (fr.status != ABCMB_OK) return fr.status;
    emu::run_cta(0, 0, 32, [&] {
        RowAcc acc;
        acc.j = -1;
        bwd(R.c, R.mb, Sinks{recbar, &acc}, fr, Sb);
    });
    return ABCMB_OK;
}
