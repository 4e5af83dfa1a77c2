// Background and perturbation kernels plus the option helpers of the C ABI
// (include/abcmb.h).
//
// background_kernel: one warp per cosmology runs abcmb::build_background.
// perturb_quad_kernel (abcmb_ode_quad.cuh): four lanes per (cosmology, k)
// mode (eight for the modes of the highest k, abcmb_options.n_wide), state in
// registers and shared memory; the path for hierarchies up to kQLmax = 63.
// perturb_kernel: one thread per mode runs abcmb::integrate_mode with the
// per-mode working vectors in a global workspace, laid out
// [vector][component][mode] so that the lanes of a warp touch consecutive
// addresses; the path for hierarchies 64..kLmaxHier, whose state does not fit
// on chip.
// Both order modes k-descending, so that the most expensive modes are
// scheduled first and a warp's modes share one k across cosmologies.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "abcmb_launch.cuh"
#include "abcmb_ode_quad.cuh"

namespace abcmb {

// one warp (32 threads) per cosmology
__global__ void __launch_bounds__(32) background_kernel(int B, const double *__restrict__ params, double *bg,
                                                         long len, int n_tau, double m_ncdm, int node_recipe)
{
    const int b = blockIdx.x;
    if (b >= B) return;
    build_background(params + (long)b * ABCMB_NPARAM, bg + (long)b * len, n_tau, threadIdx.x, 32, m_ncdm,
                     node_recipe);
}

constexpr int kLmaxHier = 128;

__global__ void __launch_bounds__(64)
perturb_kernel(int B, int Nk, const double *__restrict__ bg, long len, const double *__restrict__ kv,
               int Lg, int Lp, int Ln, double rtol, double atol, int max_steps, double s_sw,
               double s_isw, double s_dop, double *S, int *status, int *steps, double *work)
{
    __shared__ double sa[kLmaxHier + 1], sb[kLmaxHier + 1];
    for (int l = threadIdx.x; l <= kLmaxHier; l += blockDim.x) {
        sa[l] = (double)l / (2.0 * l + 1.0);
        sb[l] = (l + 1.0) / (2.0 * l + 1.0);
    }
    __syncthreads();
    const long M = (long)B * Nk;
    const long mi = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= M) return;
    const int kidx = Nk - 1 - (int)(mi / B);
    const int b = (int)(mi % B);
    const OdeDims d = ode_dims(Lg, Lp, Ln);
    const StreamCoef sc = {sa, sb};
    const double *rec = bg + (long)b * len;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    const double sw[3] = {s_sw, s_isw, s_dop};
    double *Sm = S + ((long)b * Nk + kidx) * (long)n_tau * 3;
    ModeResult r;
    if (rec[ABCMB_S_STATUS] != 0.0) {
        r.status = ABCMB_E_NONFINITE;
        r.steps = 0;
        r.substeps = 0;
        for (int n = 0; n < 3 * n_tau; n++) Sm[n] = 0.0;
    } else {
        r = integrate_mode(d, sc, rec, kv[kidx], rtol, atol, max_steps, sw, work + mi, M, Sm);
    }
    status[(long)b * Nk + kidx] = r.status;
    if (steps) {
        steps[2 * ((long)b * Nk + kidx)] = r.steps;
        steps[2 * ((long)b * Nk + kidx) + 1] = r.substeps;
    }
}

static int max_hier(const abcmb_options *o)
{
    int L = o->lmax_g;
    if (o->lmax_pol > L) L = o->lmax_pol;
    if (o->lmax_nu > L) L = o->lmax_nu;
    return L;
}

template <int P>
static int launch_quad(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                       int *st, int *steps, cudaStream_t s)
{
    constexpr int W = 1; // one warp per CTA: fine-grained scheduling of uneven modes
    const size_t smem = W * quad_smem_per_warp<P>();
    auto kern = perturb_quad_kernel<P, W>;
    const long avail = smem_optin((const void *)kern);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long M = (long)B * Nk;
    // the highest k on eight lanes per mode (four modes per warp); P = 4 keeps
    // four lanes (lane 0 must hold l <= 2)
    long kw = P >= 8 ? o->n_wide : 0;
    if (kw > Nk) kw = Nk;
    const long M8 = (long)B * kw;
    const long nb8 = (M8 + 3) / 4, blocks = nb8 + (M - M8 + 8 * W - 1) / (8 * W);
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    const long len = (long)ABCMB_BG_LEN(o->n_tau);
    kern<<<(unsigned)blocks, 32 * W, smem, s>>>(B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->rtol,
                                                 o->atol, o->max_steps, o->scale_sw, o->scale_isw, o->scale_dop, S,
                                                 st, steps, (int)nb8, M8, o->err_floor);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

static int perturb_on_chip(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                           int *st, int *steps, cudaStream_t s)
{
    const int L = max_hier(o);
    if (L <= 15) return launch_quad<4>(B, bg, k, Nk, o, S, st, steps, s);
    if (L <= 31) return launch_quad<8>(B, bg, k, Nk, o, S, st, steps, s);
    return launch_quad<16>(B, bg, k, Nk, o, S, st, steps, s);
}

static int perturb_in_workspace(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                double *S, int *st, int *steps, double *work, cudaStream_t s)
{
    const long len = (long)ABCMB_BG_LEN(o->n_tau);
    const long M = (long)B * Nk;
    const int threads = 64;
    const long blocks = (M + threads - 1) / threads;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    perturb_kernel<<<(unsigned)blocks, threads, 0, s>>>(B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu,
                                                         o->rtol, o->atol, o->max_steps, o->scale_sw, o->scale_isw,
                                                         o->scale_dop, S, st, steps, work);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

} // namespace abcmb

// ---------------------------------------------------------------- C ABI
extern "C" void abcmb_default_options(abcmb_options *o)
{
    o->lmax_g = 12;
    o->lmax_pol = 12;
    o->lmax_nu = 12;
    o->lmax_cl = 2500;
    o->n_tau = 6000;
    o->max_steps = 2000000;
    o->rtol = 1e-6;
    o->atol = 1e-12;
    o->scale_sw = o->scale_isw = o->scale_dop = o->scale_pol = 1.0;
    o->m_ncdm = 0.0;
    o->lmax_ncdm = 0;
    o->node_recipe = 0;
    o->n_wide = 0;
    o->err_floor = 1e-4;
}

extern "C" int abcmb_validate_options(const abcmb_options *o)
{
    if (!o) return ABCMB_E_INVALID_ARG;
    if (o->lmax_g < 4 || o->lmax_g > abcmb::kLmaxHier || o->lmax_pol < 4 || o->lmax_pol > abcmb::kLmaxHier ||
        o->lmax_nu < 4 || o->lmax_nu > abcmb::kLmaxHier)
        return ABCMB_E_INVALID_ARG;
    if (o->lmax_cl < 2 || o->lmax_cl > 5000) return ABCMB_E_INVALID_ARG;
    if (o->n_tau < 8 || o->n_tau > 65536) return ABCMB_E_INVALID_ARG;
    if (o->max_steps < 1) return ABCMB_E_INVALID_ARG;
    if (!(o->rtol > 0.0 && o->rtol < 1.0) || !(o->atol >= 0.0)) return ABCMB_E_INVALID_ARG;
    if (!(o->m_ncdm >= 0.0 && o->m_ncdm <= 100.0)) return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm == 0.0 ? o->lmax_ncdm != 0 : (o->lmax_ncdm < 3 || o->lmax_ncdm > abcmb::kQLmax))
        return ABCMB_E_INVALID_ARG;
    if (o->node_recipe != 0 && o->node_recipe != 1) return ABCMB_E_INVALID_ARG;
    if (o->n_wide < 0) return ABCMB_E_INVALID_ARG;
    if (!(o->err_floor > 0.0 && o->err_floor <= 1.0)) return ABCMB_E_INVALID_ARG;
    return ABCMB_OK;
}

namespace abcmb {
size_t perturb_warp_bytes(int B, int Nk, const abcmb_options *o);
int launch_perturb_warp(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                        int *mode_status, int *steps, double *work, cudaStream_t s);

template <int P>
static int launch_pk(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double x_out,
                     double *Pk, int *st, int *steps, cudaStream_t s)
{
    const size_t smem = quad_smem_per_warp<P>();
    auto kern = pk_quad_kernel<P>;
    const long avail = smem_optin((const void *)kern);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long blocks = ((long)B * Nk + 7) / 8;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    const long len = (long)ABCMB_BG_LEN(o->n_tau);
    kern<<<(unsigned)blocks, 32, smem, s>>>(B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->rtol, o->atol,
                                            o->max_steps, x_out, Pk, st, steps, o->err_floor);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
} // namespace abcmb

extern "C" int abcmb_matter_pk(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double z,
                               double *Pk, int *mode_status, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !Pk || !mode_status || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (!(z >= 0.0 && z <= 1000.0)) return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG; // massless neutrinos only
    const int L = abcmb::max_hier(o);
    if (L > abcmb::kQLmax) return ABCMB_E_INVALID_ARG;
    const double x_out = -log1p(z);
    cudaStream_t s = (cudaStream_t)stream;
    if (L <= 15) return abcmb::launch_pk<4>(B, bg, k, Nk, o, x_out, Pk, mode_status, nullptr, s);
    if (L <= 31) return abcmb::launch_pk<8>(B, bg, k, Nk, o, x_out, Pk, mode_status, nullptr, s);
    return abcmb::launch_pk<16>(B, bg, k, Nk, o, x_out, Pk, mode_status, nullptr, s);
}

namespace abcmb {
template <int P>
static int launch_dm(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *Dm, int *st,
                     cudaStream_t s)
{
    const size_t smem = quad_smem_per_warp<P>();
    auto kern = dm_quad_kernel<P>;
    const long avail = smem_optin((const void *)kern);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long blocks = ((long)B * Nk + 7) / 8;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    const long len = (long)ABCMB_BG_LEN(o->n_tau);
    kern<<<(unsigned)blocks, 32, smem, s>>>(B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->rtol, o->atol,
                                            o->max_steps, Dm, st, o->err_floor);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
} // namespace abcmb

extern "C" int abcmb_delta_m_nodes(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                   double *Dm, int *mode_status, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !Dm || !mode_status || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG; // massless neutrinos only
    const int L = abcmb::max_hier(o);
    if (L > abcmb::kQLmax) return ABCMB_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (L <= 15) return abcmb::launch_dm<4>(B, bg, k, Nk, o, Dm, mode_status, s);
    if (L <= 31) return abcmb::launch_dm<8>(B, bg, k, Nk, o, Dm, mode_status, s);
    return abcmb::launch_dm<16>(B, bg, k, Nk, o, Dm, mode_status, s);
}

extern "C" size_t abcmb_bg_doubles(const abcmb_options *o)
{
    if (abcmb_validate_options(o) != ABCMB_OK) return 0;
    return (size_t)ABCMB_BG_LEN(o->n_tau);
}

extern "C" size_t abcmb_perturb_workspace_bytes(int B, int Nk, const abcmb_options *o)
{
    if (B < 1 || Nk < 1 || abcmb_validate_options(o) != ABCMB_OK) return 0;
    if (o->m_ncdm > 0.0) return abcmb::perturb_warp_bytes(B, Nk, o);
    if (abcmb::max_hier(o) <= abcmb::kQLmax) return 0; // state on chip
    const abcmb::OdeDims d = abcmb::ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu);
    return (size_t)abcmb::kNvec * d.N * (size_t)B * Nk * sizeof(double);
}

extern "C" int abcmb_background_tables(int B, const double *params, const abcmb_options *o, double *bg,
                                       void *stream)
{
    if (B < 1 || !params || !bg || abcmb_validate_options(o) != ABCMB_OK) return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    abcmb::background_kernel<<<B, 32, 0, (cudaStream_t)stream>>>(B, params, bg, len, o->n_tau, o->m_ncdm,
                                                                  o->node_recipe);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

// ---------------------------------------------------------------- no-alloc variant
// Scratch of abcmb_perturb_noalloc: the perturbation kernel's working vectors
// live in this file-scope device array instead of a caller-provided
// workspace.  Every GPU that loads the library holds it until the process
// exits.  Host code may not pass the symbol itself to a kernel (on the host it
// names a stand-in, not device memory); the device address is looked up with
// cudaGetSymbolAddress, with the device current, once per device context.
static __device__ __align__(256) double g_noalloc_scratch[ABCMB_NOALLOC_SCRATCH_BYTES / sizeof(double)];

static std::mutex g_noalloc_mutex;
struct NoallocSlot {
    unsigned long long ctx_id; // the context the address belongs to (0: none yet)
    double *ptr;
};
static NoallocSlot g_noalloc_slot[256];

// Unique id of the calling thread's current context, 0 if it has none.  The
// symbol's address belongs to the context that loaded the module, so a reset
// device (a new primary context) needs a fresh lookup.
static unsigned long long current_ctx_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    if (!get_cur || !get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_cur, 4000, cudaEnableDefault, &q1) !=
                cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess || q2 != cudaDriverEntryPointSuccess) {
            get_cur = nullptr;
            get_id = nullptr;
            return 0;
        }
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static int noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return ABCMB_E_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocSlot &slot = g_noalloc_slot[dev];
    const unsigned long long id = current_ctx_id();
    if (!slot.ptr || id == 0 || id != slot.ctx_id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ABCMB_E_CUDA;
        slot.ptr = (double *)p;
        slot.ctx_id = current_ctx_id(); // the lookup makes the device's context current
    }
    *out = slot.ptr;
    return ABCMB_OK;
}

extern "C" int abcmb_perturb_noalloc(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                     double *S, int *mode_status, int *steps, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !S || !mode_status || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG; // the massive-neutrino path needs a caller's workspace
    const cudaStream_t s = (cudaStream_t)stream;
    if (abcmb::max_hier(o) <= abcmb::kQLmax) return abcmb::perturb_on_chip(B, bg, k, Nk, o, S, mode_status, steps, s);
    const size_t need = abcmb_perturb_workspace_bytes(B, Nk, o);
    if (need == 0) return ABCMB_E_INVALID_ARG;
    if (need > ABCMB_NOALLOC_SCRATCH_BYTES) return ABCMB_E_SCRATCH_TOO_SMALL;
    double *scratch = nullptr;
    const int rc = noalloc_scratch(&scratch);
    if (rc != ABCMB_OK) return rc;
    // the kernel writes every scratch element it reads, so nothing needs clearing
    return abcmb::perturb_in_workspace(B, bg, k, Nk, o, S, mode_status, steps, scratch, s);
}

extern "C" int abcmb_perturb(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                             double *S, int *mode_status, int *steps, void *workspace, size_t workspace_bytes,
                             void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !S || !mode_status || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    if (o->m_ncdm > 0.0) {
        if (!workspace || workspace_bytes < abcmb_perturb_workspace_bytes(B, Nk, o)) return ABCMB_E_INVALID_ARG;
        if (((size_t)workspace & 255) != 0) return ABCMB_E_INVALID_ARG;
        return abcmb::launch_perturb_warp(B, bg, k, Nk, o, S, mode_status, steps, (double *)workspace, s);
    }
    if (abcmb::max_hier(o) <= abcmb::kQLmax) return abcmb::perturb_on_chip(B, bg, k, Nk, o, S, mode_status, steps, s);
    if (!workspace || workspace_bytes < abcmb_perturb_workspace_bytes(B, Nk, o)) return ABCMB_E_INVALID_ARG;
    if (((size_t)workspace & 255) != 0) return ABCMB_E_INVALID_ARG;
    return abcmb::perturb_in_workspace(B, bg, k, Nk, o, S, mode_status, steps, (double *)workspace, s);
}
