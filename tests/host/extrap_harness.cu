// Host evaluation of the four-lane ODE kernel's extrapolation tables
// (abcmb_ode_quad.cuh: ExtTab and the 1/n table), for the CPU tests.
#include "abcmb_ode_quad.cuh"

using namespace abcmb;

// lam, mu: [2][kQK + 1][kQK + 1]; inv: [2 kQK + 1]; returns kQK
extern "C" int h_ext_tables(double *lam, double *mu, double *inv)
{
    const ExtTab t = make_ext();
    const InvTab v = make_inv();
    for (int g = 0; g < 2; g++)
        for (int j = 0; j <= kQK; j++)
            for (int i = 0; i <= kQK; i++) {
                lam[(g * (kQK + 1) + j) * (kQK + 1) + i] = t.lam[g][j][i];
                mu[(g * (kQK + 1) + j) * (kQK + 1) + i] = t.mu[g][j][i];
            }
    for (int n = 0; n <= 2 * kQK; n++) inv[n] = v.inv[n];
    return kQK;
}
