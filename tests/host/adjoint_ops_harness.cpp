// Host build of the adjoint operators (abcmb_adjoint_ops.cuh) for the CPU
// tests: flat C entry points over random states, background points and node
// data supplied by the test.
#include <vector>

#include "abcmb_adjoint_ops.cuh"

using namespace abcmb;
using namespace abcmb::adj;

namespace {
struct Ctx {
    OdeDims d;
    double a[129], b[129];
    StreamCoef sc;
};
Ctx make(int L)
{
    Ctx c;
    c.d = ode_dims(L, L, L);
    for (int l = 0; l < 129; l++) {
        c.a[l] = (double)l / (2.0 * l + 1.0);
        c.b[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    c.sc = StreamCoef{c.a, c.b};
    return c;
}
Bg10 bg(const double *p)
{
    Bg10 b;
    for (int q = 0; q < B_N; q++) b.v[q] = p[q];
    return b;
}
} // namespace

extern "C" int h_nstate(int L) { return ode_dims(L, L, L).N; }

// which: 0 E, 1 E^T, 2 T, 3 T^T, 4 solve_M, 5 solve_Mt
extern "C" void h_apply(int which, int L, double k, const double *bp, double h, const double *in, double *out)
{
    Ctx c = make(L);
    const Bg10 b = bg(bp);
    const int N = c.d.N;
    std::vector<double> x(in, in + N);
    for (int i = 0; i < N; i++) out[i] = 0.0;
    Vec vi{x.data(), 1}, vo{out, 1};
    switch (which) {
    case 0: op_E(c.d, c.sc, k, b, vi, vo, 1.0); break;
    case 1: op_Et(c.d, c.sc, k, b, vi, vo, 1.0); break;
    case 2: op_T(c.d, k, b, vi, vo, 1.0); break;
    case 3: op_Tt(c.d, k, b, vi, vo, 1.0); break;
    case 4: solve_M(c.d, k, b, h, vi); for (int i = 0; i < N; i++) out[i] = x[i]; break;
    case 5: solve_Mt(c.d, k, b, h, vi); for (int i = 0; i < N; i++) out[i] = x[i]; break;
    }
}

// which: 0 E, 1 T; bb[10] = d(v^T X(b) y)/db
extern "C" void h_bgrad(int which, int L, double k, const double *bp, const double *v, const double *y, double *bbo)
{
    Ctx c = make(L);
    const Bg10 b = bg(bp);
    std::vector<double> vv(v, v + c.d.N), yy(y, y + c.d.N);
    Bg10 bb;
    for (int q = 0; q < B_N; q++) bb.v[q] = 0.0;
    if (which == 0) op_E_bgrad(c.d, c.sc, k, b, Vec{vv.data(), 1}, Vec{yy.data(), 1}, 1.0, bb);
    else op_T_bgrad(c.d, k, Vec{vv.data(), 1}, Vec{yy.data(), 1}, 1.0, bb);
    for (int q = 0; q < B_N; q++) bbo[q] = bb.v[q];
}

extern "C" void h_sources(int L, double k, const double *bp, const double *np, const double *sw, const double *y,
                          double *S)
{
    Ctx c = make(L);
    std::vector<double> yy(y, y + c.d.N);
    const NodeD n{np[0], np[1], np[2], np[3], np[4]};
    sources_fwd(c.d, k, bg(bp), n, sw, Vec{yy.data(), 1}, S);
}

extern "C" void h_sources_rev(int L, double k, const double *bp, const double *np, const double *sw, const double *y,
                              const double *Sb, double *yb, double *bbo, double *nbo)
{
    Ctx c = make(L);
    std::vector<double> yy(y, y + c.d.N);
    for (int i = 0; i < c.d.N; i++) yb[i] = 0.0;
    const NodeD n{np[0], np[1], np[2], np[3], np[4]};
    Bg10 bb;
    for (int q = 0; q < B_N; q++) bb.v[q] = 0.0;
    NodeD nb{0, 0, 0, 0, 0};
    sources_rev(c.d, k, bg(bp), n, sw, Vec{yy.data(), 1}, Sb, Vec{yb, 1}, bb, nb);
    for (int q = 0; q < B_N; q++) bbo[q] = bb.v[q];
    nbo[0] = nb.Hc;
    nbo[1] = nb.dHc;
    nbo[2] = nb.g;
    nbo[3] = nb.dg;
    nbo[4] = nb.emk;
}

extern "C" void h_initial(int L, double k, double tau_i, double Rn, double *y)
{
    Ctx c = make(L);
    initial_fwd(c.d, k, tau_i, Rn, Vec{y, 1});
}

extern "C" double h_initial_d(int which, int L, double k, double tau_i, double Rn, const double *yb)
{
    Ctx c = make(L);
    std::vector<double> v(yb, yb + c.d.N);
    return which == 0 ? initial_dtau(c.d, k, tau_i, Rn, Vec{v.data(), 1})
                      : initial_dRn(c.d, k, tau_i, Rn, Vec{v.data(), 1});
}
