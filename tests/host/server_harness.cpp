// Host build of the spectrum server's runtime (abcmb_server.cu, compiled as
// C++ beside this file) for the CPU tests, over the stand-in CUDA runtime of
// tests/host/fake_cuda/cuda_runtime.h and stand-ins for the library calls the
// server makes.  The stand-in compute writes, for each cosmology of a batch,
// C_l values that identify the request (its first parameter), the spectrum,
// l, its k-grid size and largest k, and sets the background or mode status a
// request asks for through its parameters; every device pointer the server
// hands over is checked to lie in the caller's arena, and the spans of
// batches in flight at the same time never to overlap.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <vector>

#include "abcmb.h"

struct FakeStream {
    int id;
};
struct FakeEvent {
    FakeStream *stream = nullptr;
    int pending = 0;
};

namespace {
int g_not_ready = 2; // answers of "not ready" after each record
int g_streams = 0;
const char *g_lo = nullptr, *g_hi = nullptr; // the arena
int g_violations = 0;
struct Span {
    const char *lo, *hi;
    FakeStream *s;
};
std::vector<Span> g_inflight;
int g_max_inflight = 0;
struct Launch {
    int B, lmax_cl, n_k, stream;
    long long tag[8];
};
std::vector<Launch> g_launches;

void in_arena(const void *p, size_t bytes)
{
    const char *c = (const char *)p;
    if (!(c >= g_lo && c + bytes <= g_hi)) g_violations++;
}

const long kTagSlot = 60, kFailSlot = 61; // spare scalar slots of a record
} // namespace

// ---- the stand-in runtime ----
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned)
{
    *s = new FakeStream{g_streams++};
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s)
{
    delete s;
    return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned)
{
    *e = new FakeEvent;
    return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t e)
{
    delete e;
    return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s)
{
    e->stream = s;
    e->pending = g_not_ready;
    return cudaSuccess;
}
cudaError_t cudaEventQuery(cudaEvent_t e)
{
    if (e->pending > 0) {
        e->pending--;
        return cudaErrorNotReady;
    }
    for (size_t i = 0; i < g_inflight.size();) // the stream's batch is done
        if (g_inflight[i].s == e->stream) g_inflight.erase(g_inflight.begin() + (long)i);
        else i++;
    return cudaSuccess;
}
cudaError_t cudaMallocHost(void **p, size_t bytes)
{
    *p = std::aligned_alloc(256, (bytes + 255) & ~(size_t)255);
    return *p ? cudaSuccess : cudaErrorUnknown;
}
cudaError_t cudaFreeHost(void *p)
{
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t)
{
    in_arena(kind == cudaMemcpyHostToDevice ? dst : src, bytes);
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
}
cudaError_t cudaMemcpy2DAsync(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                              cudaMemcpyKind kind, cudaStream_t)
{
    for (size_t r = 0; r < height; r++) {
        in_arena(kind == cudaMemcpyHostToDevice ? (char *)dst + r * dpitch : (const char *)src + r * spitch, width);
        std::memcpy((char *)dst + r * dpitch, (const char *)src + r * spitch, width);
    }
    return cudaSuccess;
}

// ---- stand-ins for the library calls the server makes ----
extern "C" int abcmb_validate_options(const abcmb_options *o)
{
    return o && o->lmax_cl >= 2 && o->lmax_cl <= 5000 && o->n_tau >= 8 && o->lmax_g >= 4 ? ABCMB_OK
                                                                                         : ABCMB_E_INVALID_ARG;
}
extern "C" size_t abcmb_bg_doubles(const abcmb_options *o)
{
    return abcmb_validate_options(o) == ABCMB_OK ? (size_t)ABCMB_BG_LEN(o->n_tau) : 0;
}
extern "C" size_t abcmb_perturb_workspace_bytes(int B, int Nk, const abcmb_options *o)
{
    const int L = o->lmax_g > o->lmax_pol ? o->lmax_g : o->lmax_pol;
    return (L > o->lmax_nu ? L : o->lmax_nu) > 63 ? (size_t)B * Nk * 8 : 0;
}
extern "C" int abcmb_background_tables(int B, const double *params, const abcmb_options *o, double *bg,
                                       void *stream)
{
    const long len = (long)abcmb_bg_doubles(o);
    in_arena(params, (size_t)B * ABCMB_NPARAM * sizeof(double));
    in_arena(bg, (size_t)B * len * sizeof(double));
    const char *lo = (const char *)bg, *hi = lo + (size_t)B * len * sizeof(double);
    for (const Span &sp : g_inflight)
        if (lo < sp.hi && sp.lo < hi) g_violations++;
    g_inflight.push_back(Span{lo, hi, (FakeStream *)stream});
    if ((int)g_inflight.size() > g_max_inflight) g_max_inflight = (int)g_inflight.size();
    Launch L{B, o->lmax_cl, 0, ((FakeStream *)stream)->id, {}};
    for (int b = 0; b < B; b++) {
        double *r = bg + b * len;
        r[ABCMB_S_STATUS] = params[b * ABCMB_NPARAM] < 0.0 ? 1.0 : 0.0; // a negative omega_b: no background
        r[kTagSlot] = params[b * ABCMB_NPARAM];
        r[kFailSlot] = params[b * ABCMB_NPARAM + 5];
        if (b < 8) L.tag[b] = (long long)params[b * ABCMB_NPARAM];
    }
    g_launches.push_back(L);
    return ABCMB_OK;
}
extern "C" int abcmb_perturb(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                             int *mode_status, int *, void *, size_t, void *)
{
    const long len = (long)abcmb_bg_doubles(o);
    in_arena(k, Nk * sizeof(double));
    in_arena(S, (size_t)B * Nk * o->n_tau * 3 * sizeof(double));
    in_arena(mode_status, (size_t)B * Nk * sizeof(int));
    g_launches.back().n_k = Nk;
    for (int b = 0; b < B; b++)
        for (int i = 0; i < Nk; i++) // tau_reio > 1: a mode out of steps
            mode_status[b * Nk + i] = bg[b * len + kFailSlot] > 1.0 ? ABCMB_E_MAX_STEPS : ABCMB_OK;
    return ABCMB_OK;
}
extern "C" int abcmb_project_mixed(int B, const double *, const double *S, const double *, int Nk,
                                   const abcmb_options *o, float *Delta, void *)
{
    in_arena(S, (size_t)B * Nk * o->n_tau * 3 * sizeof(double));
    in_arena(Delta, (size_t)B * Nk * (o->lmax_cl - 1) * 2 * sizeof(float));
    return ABCMB_OK;
}
extern "C" int abcmb_cl_mixed(int B, const double *bg, const float *Delta, const double *k, int Nk,
                              const abcmb_options *o, double *Cl, void *)
{
    const long len = (long)abcmb_bg_doubles(o), nl = o->lmax_cl - 1;
    in_arena(Delta, (size_t)B * Nk * nl * 2 * sizeof(float));
    in_arena(Cl, (size_t)B * 3 * nl * sizeof(double));
    for (int b = 0; b < B; b++)
        for (int t = 0; t < 3; t++)
            for (long q = 0; q < nl; q++)
                Cl[(b * 3 + t) * nl + q] = 1000.0 * bg[b * len + kTagSlot] + 100.0 * t + (double)q + 1e-3 * Nk +
                                           1e-6 * k[Nk - 1];
    return ABCMB_OK;
}

// ---- for the tests ----
extern "C" void h_reset(const void *arena, size_t bytes, int not_ready)
{
    g_lo = (const char *)arena;
    g_hi = g_lo + bytes;
    g_not_ready = not_ready;
    g_violations = 0;
    g_inflight.clear();
    g_max_inflight = 0;
    g_launches.clear();
}
extern "C" void *h_arena(size_t bytes) { return std::aligned_alloc(256, (bytes + 255) & ~(size_t)255); }
extern "C" void h_free(void *p) { std::free(p); }
extern "C" int h_violations() { return g_violations; }
extern "C" int h_max_inflight() { return g_max_inflight; }
extern "C" int h_launches() { return (int)g_launches.size(); }
// launch i: B, lmax_cl, n_k, stream id, and the first parameters (tags) of its requests
extern "C" void h_launch(int i, int *info, long long *tags)
{
    const Launch &L = g_launches[i];
    info[0] = L.B;
    info[1] = L.lmax_cl;
    info[2] = L.n_k;
    info[3] = L.stream;
    for (int b = 0; b < L.B && b < 8; b++) tags[b] = L.tag[b];
}
