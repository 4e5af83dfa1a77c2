// Host build of the massive-neutrino path (the background builder with one
// massive neutrino and the one-warp-per-mode forward of abcmb_adjoint.cuh, run
// with one lane) for the CPU parity tests against the oracle.
#include <vector>

#include "abcmb_adjoint.cuh"

using namespace abcmb;
using namespace abcmb::adj;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg_m(const double *p, int n_tau, double m_ncdm, double *rec)
{
    build_background(p, rec, n_tau, 0, 1, m_ncdm);
}

// the same with a tau-node recipe (0 the default placement, 1 the refined tail)
extern "C" void h_build_bg_r(const double *p, int n_tau, double m_ncdm, int recipe, double *rec)
{
    build_background(p, rec, n_tau, 0, 1, m_ncdm, recipe);
}

// sources S[n_tau][3] of one mode; hierarchies L (all three massless chains), Lm
extern "C" int h_fwd_m(const double *rec, double k, int L, int Lm, double rtol, double *S)
{
    static double a[129], b[129];
    for (int l = 0; l < 129; l++) {
        a[l] = (double)l / (2.0 * l + 1.0);
        b[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    const OdeDims d = ode_dims(L, L, L, Lm);
    std::vector<double> work((size_t)V_COUNT * d.N, 0.0);
    ModeCtx c;
    c.d = d;
    c.sc = StreamCoef{a, b};
    c.rec = rec;
    c.tab = rec + ABCMB_BG_TABLE;
    c.ot = rec + ABCMB_BG_ODETAB;
    c.nodes = rec + ABCMB_BG_NODES;
    c.k = k;
    c.sw[0] = c.sw[1] = c.sw[2] = 1.0;
    c.n_tau = (int)rec[ABCMB_S_NTAU];
    c.ncdm_x1 = rec[ABCMB_S_NCDM_X1];
    c.ncdm_pH = rec[ABCMB_S_NCDM_PREF] * rec[ABCMB_S_H0] * rec[ABCMB_S_H0];
    ModeBufs mb{work.data(), nullptr, nullptr, nullptr, 1, 0};
    return fwd_taped(c, mb, rtol, 1e-15, 20000000, S, false).status;
}
