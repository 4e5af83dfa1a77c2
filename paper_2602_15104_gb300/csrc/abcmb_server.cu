// Continuous-batching spectrum server (host runtime over the C ABI calls).
//
// Requests (one cosmology, its lmax_cl and k-grid size) queue on the host;
// progress() admits them while a stream slot is free and the caller's device
// arena has room for their buffers (first fit over a sorted free list).  The
// request at the head of the queue is admitted first, together with up to
// kMaxBatch - 1 later requests of the same shape (lmax_cl and k grid), which
// share the k grid: the slot then runs them as one batch of cosmologies, so
// that each warp of the perturbation kernel integrates one k for up to eight
// cosmologies, whose step sequences are nearly the same (the layout of the
// batched path), instead of eight different k of one cosmology, whose
// warp-uniform step loop would run at the pace of the slowest.  Per slot the
// whole path is enqueued on its stream (params and k H2D, background tables,
// FP64 perturbations, FP32 projection and k-quadrature, C_l D2H into the
// slot's pinned buffer, completion event); finished slots are retired by
// event query, never a blocking wait, releasing their arena blocks.  Batches
// in flight on different streams overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "abcmb.h"
#include "abcmb_arena.h"

namespace {

struct Request {
    long long tag;
    double params[ABCMB_NPARAM];
    int lmax_cl, n_k;
    double k_min, k_max;
    double t_submit;
};

constexpr int kMaxBatch = 8; // cosmologies per launch: one warp's modes share a k

struct Slot {
    bool busy = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Request> reqs; // the batch: same lmax_cl and k grid
    size_t off = 0, bytes = 0;
    double *host = nullptr;     // pinned: params [B][6], k; then C_l [B][3][lmax-1] and B background statuses
    int *host_status = nullptr; // pinned: mode status words [B][n_k]
    size_t host_doubles = 0;
    int launch_rc = ABCMB_OK;
};

struct Result {
    long long tag;
    int status, lmax_cl, n_k;
    std::vector<double> cl;
};

// sizes of the device buffers of a batch of B requests of one shape, in
// bytes, in allocation order
struct Layout {
    size_t bg, k, params, S, status, D, Cl, total;
};

Layout layout_of(const abcmb_options *o, int n_k, int B = 1)
{
    Layout L;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    L.bg = up((size_t)B * abcmb_bg_doubles(o) * sizeof(double));
    L.k = up((size_t)n_k * sizeof(double));
    L.params = up((size_t)B * ABCMB_NPARAM * sizeof(double));
    L.S = up((size_t)B * n_k * o->n_tau * 3 * sizeof(double));
    L.status = up((size_t)B * n_k * sizeof(int));
    L.D = up((size_t)B * n_k * (o->lmax_cl - 1) * 2 * sizeof(float));
    L.Cl = up((size_t)B * 3 * (o->lmax_cl - 1) * sizeof(double));
    L.total = L.bg + L.k + L.params + L.S + L.status + L.D + L.Cl;
    return L;
}

bool same_shape(const Request &a, const Request &b)
{
    return a.lmax_cl == b.lmax_cl && a.n_k == b.n_k && a.k_min == b.k_min && a.k_max == b.k_max;
}

} // namespace

struct abcmb_server {
    abcmb_options base;
    char *arena_base = nullptr;
    abcmb::Arena arena;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::deque<Result> results;
    int max_lmax = 0, max_nk = 0;
};

extern "C" size_t abcmb_server_request_bytes(const abcmb_options *o, int lmax_cl, int n_k)
{
    if (!o || lmax_cl < 2 || n_k < 2) return 0;
    abcmb_options r = *o;
    r.lmax_cl = lmax_cl;
    if (abcmb_validate_options(&r) != ABCMB_OK) return 0;
    return layout_of(&r, n_k).total;
}

extern "C" int abcmb_server_create(void *arena, size_t arena_bytes, int n_slots, int max_lmax_cl, int max_n_k,
                                   const abcmb_options *o, abcmb_server **out)
{
    if (!out || !arena || ((size_t)arena & 255) != 0 || n_slots < 1 || n_slots > 256 || max_n_k < 2 ||
        abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    abcmb_options r = *o;
    r.lmax_cl = max_lmax_cl;
    if (abcmb_validate_options(&r) != ABCMB_OK) return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG; // served requests use the on-chip path
    // requests run the on-chip perturbation path, which needs no workspace
    if (abcmb_perturb_workspace_bytes(1, 2, o) != 0) return ABCMB_E_INVALID_ARG;
    *out = nullptr;
    abcmb_server *s = new (std::nothrow) abcmb_server;
    if (!s) return ABCMB_E_INVALID_ARG;
    s->base = *o;
    s->arena_base = (char *)arena;
    s->arena.init(arena_bytes);
    s->max_lmax = max_lmax_cl;
    s->max_nk = max_n_k;
    s->slots.resize(n_slots);
    // params + k on the way in, C_l on the way out, then the background status words
    const size_t host_doubles = std::max((size_t)kMaxBatch * ABCMB_NPARAM + max_n_k,
                                         (size_t)kMaxBatch * 3 * (max_lmax_cl - 1)) + kMaxBatch;
    for (Slot &sl : s->slots) {
        sl.host_doubles = host_doubles;
        sl.reqs.reserve(kMaxBatch);
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&sl.host, host_doubles * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void **)&sl.host_status, (size_t)kMaxBatch * max_n_k * sizeof(int)) != cudaSuccess) {
            abcmb_server_destroy(s);
            return ABCMB_E_CUDA;
        }
    }
    *out = s;
    return ABCMB_OK;
}

extern "C" int abcmb_server_destroy(abcmb_server *s)
{
    if (!s) return ABCMB_E_INVALID_ARG;
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.host_status) cudaFreeHost(sl.host_status);
    }
    delete s;
    return ABCMB_OK;
}

extern "C" int abcmb_server_submit(abcmb_server *s, long long tag, const double *params_host, int lmax_cl, int n_k,
                                   double k_min, double k_max)
{
    if (!s || !params_host || lmax_cl < 2 || lmax_cl > s->max_lmax || n_k < 2 || n_k > s->max_nk ||
        !(k_min > 0.0) || !(k_max > k_min))
        return ABCMB_E_INVALID_ARG;
    abcmb_options r = s->base;
    r.lmax_cl = lmax_cl;
    if (layout_of(&r, n_k).total > s->arena.size()) return ABCMB_E_SCRATCH_TOO_SMALL;
    Request q;
    q.tag = tag;
    memcpy(q.params, params_host, sizeof(q.params));
    q.lmax_cl = lmax_cl;
    q.n_k = n_k;
    q.k_min = k_min;
    q.k_max = k_max;
    q.t_submit = 0.0;
    s->queue.push_back(q);
    return ABCMB_OK;
}

static int launch(abcmb_server *s, Slot &sl)
{
    const Request &q = sl.reqs[0];
    const int B = (int)sl.reqs.size();
    abcmb_options o = s->base;
    o.lmax_cl = q.lmax_cl;
    const Layout L = layout_of(&o, q.n_k, B);
    char *p = s->arena_base + sl.off;
    double *bg = (double *)p;
    double *k = (double *)(p + L.bg);
    double *params = (double *)(p + L.bg + L.k);
    double *S = (double *)(p + L.bg + L.k + L.params);
    int *st = (int *)(p + L.bg + L.k + L.params + L.S);
    float *D = (float *)(p + L.bg + L.k + L.params + L.S + L.status);
    double *Cl = (double *)(p + L.bg + L.k + L.params + L.S + L.status + L.D);
    // host staging: params of each cosmology, then log-spaced k (the workload's grid rule)
    double *h = sl.host;
    for (int b = 0; b < B; b++) memcpy(h + b * ABCMB_NPARAM, sl.reqs[b].params, sizeof(q.params));
    double *hk = h + B * ABCMB_NPARAM;
    const double l0 = std::log(q.k_min), l1 = std::log(q.k_max);
    for (int i = 0; i < q.n_k; i++) hk[i] = std::exp(l0 + (l1 - l0) * i / (q.n_k - 1));
    cudaStream_t st_ = sl.stream;
    if (cudaMemcpyAsync(params, h, (size_t)B * ABCMB_NPARAM * sizeof(double), cudaMemcpyHostToDevice, st_) !=
            cudaSuccess ||
        cudaMemcpyAsync(k, hk, q.n_k * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
        return ABCMB_E_CUDA;
    int rc = abcmb_background_tables(B, params, &o, bg, st_);
    if (rc == ABCMB_OK) rc = abcmb_perturb(B, bg, k, q.n_k, &o, S, st, nullptr, nullptr, 0, st_);
    if (rc == ABCMB_OK) rc = abcmb_project_mixed(B, bg, S, k, q.n_k, &o, D, st_);
    if (rc == ABCMB_OK) rc = abcmb_cl_mixed(B, bg, D, k, q.n_k, &o, Cl, st_);
    if (rc != ABCMB_OK) return rc;
    // the host staging buffer is reused for C_l only after the H2D copies ran (stream order)
    const size_t ncl = 3 * (size_t)(q.lmax_cl - 1), len = abcmb_bg_doubles(&o);
    if (cudaMemcpyAsync(h, Cl, B * ncl * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess ||
        cudaMemcpyAsync(sl.host_status, st, (size_t)B * q.n_k * sizeof(int), cudaMemcpyDeviceToHost, st_) !=
            cudaSuccess ||
        cudaMemcpy2DAsync(h + sl.host_doubles - kMaxBatch, sizeof(double), bg + ABCMB_S_STATUS,
                          len * sizeof(double), sizeof(double), B, cudaMemcpyDeviceToHost, st_) != cudaSuccess ||
        cudaEventRecord(sl.done, st_) != cudaSuccess)
        return ABCMB_E_CUDA;
    return ABCMB_OK;
}

// Admit, launch and retire without blocking; returns the number of requests
// in flight afterwards (>= 0) or a negative error code.
extern "C" int abcmb_server_progress(abcmb_server *s)
{
    if (!s) return -ABCMB_E_INVALID_ARG;
    // retire
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        const int B = (int)sl.reqs.size();
        for (int b = 0; b < B; b++) {
            const Request &q = sl.reqs[b];
            Result r;
            r.tag = q.tag;
            r.lmax_cl = q.lmax_cl;
            r.n_k = q.n_k;
            r.status = ABCMB_OK;
            if (e != cudaSuccess || sl.launch_rc != ABCMB_OK) {
                r.status = sl.launch_rc != ABCMB_OK ? sl.launch_rc : ABCMB_E_CUDA;
            } else {
                const size_t ncl = 3 * (size_t)(q.lmax_cl - 1);
                if (sl.host[sl.host_doubles - kMaxBatch + b] != 0.0) r.status = ABCMB_E_BACKGROUND;
                for (int i = 0; i < q.n_k; i++)
                    if (sl.host_status[(size_t)b * q.n_k + i] != ABCMB_OK) r.status = sl.host_status[(size_t)b * q.n_k + i];
                r.cl.assign(sl.host + b * ncl, sl.host + (b + 1) * ncl);
            }
            s->results.push_back(std::move(r));
        }
        s->arena.release(sl.off, sl.bytes);
        sl.reqs.clear();
        sl.busy = false;
    }
    // admit: the head of the queue first, with the later requests of its shape
    while (!s->queue.empty()) {
        Slot *free_slot = nullptr;
        for (Slot &sl : s->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        if (!free_slot) break;
        const Request head = s->queue.front();
        size_t pick[kMaxBatch];
        int n = 0;
        for (size_t i = 0; i < s->queue.size() && n < kMaxBatch; i++)
            if (same_shape(s->queue[i], head)) pick[n++] = i;
        abcmb_options o = s->base;
        o.lmax_cl = head.lmax_cl;
        size_t off = 0, bytes = 0;
        int B = n;
        for (; B >= 1; B--) { // the largest batch the arena holds now
            bytes = layout_of(&o, head.n_k, B).total;
            if (s->arena.alloc(bytes, &off)) break;
        }
        if (B < 1) break; // wait for memory: the head keeps its place
        free_slot->reqs.clear();
        for (int j = 0; j < B; j++) free_slot->reqs.push_back(s->queue[pick[j]]);
        for (int j = B - 1; j >= 0; j--) s->queue.erase(s->queue.begin() + (long)pick[j]);
        free_slot->off = off;
        free_slot->bytes = bytes;
        free_slot->busy = true;
        free_slot->launch_rc = launch(s, *free_slot);
        if (free_slot->launch_rc != ABCMB_OK) cudaEventRecord(free_slot->done, free_slot->stream);
    }
    int n = 0;
    for (const Slot &sl : s->slots) n += sl.busy ? (int)sl.reqs.size() : 0;
    return n;
}

extern "C" int abcmb_server_queued(const abcmb_server *s) { return s ? (int)s->queue.size() : -1; }

// Pop one finished request: 1 and its tag, status and C_l [3][lmax_cl - 1]
// (TT, TE, EE) into cl_host (room for cl_capacity doubles), or 0 if none is
// ready.  A result that does not fit stays queued and ABCMB_E_INVALID_ARG is
// returned negated.
extern "C" int abcmb_server_poll(abcmb_server *s, long long *tag, int *status, int *lmax_cl, double *cl_host,
                                 size_t cl_capacity)
{
    if (!s || !tag || !status || !lmax_cl || !cl_host) return -ABCMB_E_INVALID_ARG;
    if (s->results.empty()) return 0;
    Result &r = s->results.front();
    if (r.cl.size() > cl_capacity) return -ABCMB_E_INVALID_ARG;
    *tag = r.tag;
    *status = r.status;
    *lmax_cl = r.lmax_cl;
    if (!r.cl.empty()) memcpy(cl_host, r.cl.data(), r.cl.size() * sizeof(double));
    s->results.pop_front();
    return 1;
}
