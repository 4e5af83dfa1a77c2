// Host build of the library's lensing math (abcmb_lensing.cuh) for the CPU
// parity tests against the oracle: the per-node correlation functions and the
// back transform, summed serially over the Gauss-Legendre nodes.
#include <cmath>
#include <vector>

#include "abcmb_lensing.cuh"

using namespace abcmb::lens;

// Cl [3][L-1] (TT, TE, EE for l = 2..L), Cpsi [L-1]; out [4][lout-1]: TT, TE, EE, BB
extern "C" void h_lens(const double *Cl, const double *Cpsi, int L, int lout, int n_mu, double *out)
{
    LensIn in{Cl, Cl + 2 * (L - 1), Cl + (L - 1), Cpsi, L};
    const double cgl1 = cgl_at_one(in);
    std::vector<double> acc(4 * (size_t)(lout + 1), 0.0);
    for (int i = 0; i < n_mu; i++) {
        double mu, w, x[4];
        gauss_legendre(n_mu, i, &mu, &w);
        corr_at(mu, in, cgl1, x);
        DSeq d00 = dseq_init(0, 0, mu), d22 = dseq_init(2, 2, mu), d2m2 = dseq_init(2, -2, mu),
             d20 = dseq_init(2, 0, mu);
        for (int l = 0; l <= lout; l++) {
            const double f = 2.0 * kPi * w;
            acc[0 * (lout + 1) + l] += f * x[0] * dval(d00, l);
            acc[1 * (lout + 1) + l] += f * x[1] * dval(d22, l);
            acc[2 * (lout + 1) + l] += f * x[2] * dval(d2m2, l);
            acc[3 * (lout + 1) + l] += f * x[3] * dval(d20, l);
            dadvance(d00, l, mu);
            dadvance(d22, l, mu);
            dadvance(d2m2, l, mu);
            dadvance(d20, l, mu);
        }
    }
    const int nl = lout - 1;
    for (int l = 2; l <= lout; l++) {
        const double dT = acc[l], dP = acc[(lout + 1) + l], dM = acc[2 * (lout + 1) + l], dX = acc[3 * (lout + 1) + l];
        out[l - 2] = Cl[l - 2] + dT;
        out[nl + l - 2] = Cl[(L - 1) + l - 2] + dX;
        out[2 * nl + l - 2] = Cl[2 * (L - 1) + l - 2] + 0.5 * (dP + dM);
        out[3 * nl + l - 2] = 0.5 * (dP - dM);
    }
}

// Limber C_l^psi for l = 2..lmax: nodes [n_tau][8] as the background record's
// node table, dm [Nk][n_tau]; out [lmax-1]
extern "C" void h_cl_psi(const double *nodes, int n_tau, double tau0, double Om_m, double H0, const double *dm,
                         const double *kv, int Nk, double As, double ns, int lmax, double *out)
{
    std::vector<double> chi(n_tau, 0.0), coef(n_tau, 0.0);
    const int is = limber_prepare(nodes, n_tau, tau0, Om_m, H0, chi.data(), coef.data());
    for (int l = 2; l <= lmax; l++) out[l - 2] = limber_cl_at(l, chi.data(), coef.data(), is, n_tau, dm, kv, Nk, As, ns);
}
