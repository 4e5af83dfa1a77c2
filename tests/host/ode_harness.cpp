// Host build of the thread-per-mode perturbation solver (abcmb_ode.cuh, the
// path for hierarchies above 63) for the CPU parity tests against the oracle.
#include <thread>
#include <vector>

#include "abcmb_ode.cuh"

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

// sources S[n_tau][3] of one mode with all three hierarchies at L; returns the status
extern "C" int h_integrate(const double *rec, double k, int L, double rtol, double *S, int *steps)
{
    static double a[129], b[129]; // l = 0..128, the deepest hierarchy
    for (int l = 0; l <= 128; l++) {
        a[l] = (double)l / (2.0 * l + 1.0);
        b[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    const OdeDims d = ode_dims(L, L, L);
    std::vector<double> work((size_t)kNvec * d.N, 0.0);
    const double sw[3] = {1.0, 1.0, 1.0};
    const ModeResult r = integrate_mode(d, StreamCoef{a, b}, rec, k, rtol, 1e-12, 2000000, sw, work.data(), 1, S);
    steps[0] = r.steps;
    steps[1] = r.substeps;
    return r.status;
}

// M modes of one record at once, as perturb_kernel lays them out: one host
// thread per mode, the working vectors of all modes interleaved in one
// workspace (element e of mode m at e * M + m); S[M][n_tau][3], status[M]
extern "C" void h_integrate_batch(const double *rec, const double *k, int M, int L, double rtol, double *S,
                                  int *status)
{
    static double a[129], b[129];
    for (int l = 0; l <= 128; l++) {
        a[l] = (double)l / (2.0 * l + 1.0);
        b[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    const OdeDims d = ode_dims(L, L, L);
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    std::vector<double> work((size_t)kNvec * d.N * M, 0.0);
    const double sw[3] = {1.0, 1.0, 1.0};
    std::vector<std::thread> th;
    for (int m = 0; m < M; m++)
        th.emplace_back([&, m] {
            const ModeResult r = integrate_mode(d, StreamCoef{a, b}, rec, k[m], rtol, 1e-12, 2000000, sw,
                                                work.data() + m, M, S + (size_t)m * n_tau * 3);
            status[m] = r.status;
        });
    for (auto &t : th) t.join();
}
