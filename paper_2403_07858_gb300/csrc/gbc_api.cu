// Host side of the C ABI declared in include/gbc.h: contexts, graph loading
// (validation and per-side index build on the device) and the count pipeline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbc.h"
#include "gbc_internal.cuh"

using namespace gbc;

// ---------------------------------------------------------------------------
// errors
static thread_local char t_err[512] = "";

static gbc_status fail(gbc_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof t_err, fmt, ap);
    va_end(ap);
    return s;
}

void gbc::set_last_error(const char *msg) { snprintf(t_err, sizeof t_err, "%s", msg); }

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            gbc_status s_ = (e_ == cudaErrorMemoryAllocation) ? GBC_ERR_OOM : GBC_ERR_CUDA;   \
            return fail(s_, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                     \
    } while (0)

constexpr int kAuxStreams = 8;

struct TuneKey {
    const void *graph;
    int p, q;
    bool operator<(const TuneKey &o) const {
        return graph != o.graph ? graph < o.graph : (p != o.p ? p < o.p : q < o.q);
    }
};

// A stream with its auxiliary streams: the counts of one pipeline run on it.
struct Lane {
    cudaStream_t st = nullptr;
    cudaStream_t aux[kAuxStreams] = {};      // per-job launches of a batch overlap on these
    cudaEvent_t fork_ev = nullptr, join_ev[kAuxStreams] = {};
    DoneRec *done_h = nullptr;               // host-mapped completion records of a batch
    DoneRec *done_d = nullptr;               // the same records as device pointers
    int done_cap = 0;
    // Completion records for n counts, zeroed (grows the mapped buffer as needed).
    cudaError_t ensure_done(int n) {
        if (n > done_cap) {
            if (done_h) cudaFreeHost(done_h);
            done_h = nullptr;
            done_cap = 0;
            const int cap = std::max(n, 64);
            cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&done_h), sizeof(DoneRec) * cap,
                                          cudaHostAllocMapped);
            if (e != cudaSuccess) { done_h = nullptr; return e; }
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&done_d), done_h, 0);
            if (e != cudaSuccess) return e;
            done_cap = cap;
        }
        memset(done_h, 0, sizeof(DoneRec) * n);
        return cudaSuccess;
    }
    cudaError_t create(cudaStream_t main) {
        st = main;
        cudaError_t e = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
        for (int i = 0; i < kAuxStreams && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&aux[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_ev[i], cudaEventDisableTiming);
        }
        return e;
    }
    void destroy() {
        for (int i = 0; i < kAuxStreams; ++i) {
            if (aux[i]) cudaStreamDestroy(aux[i]);
            if (join_ev[i]) cudaEventDestroy(join_ev[i]);
        }
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (done_h) cudaFreeHost(done_h);
        done_h = nullptr;
        done_cap = 0;
    }
};

// Exact scratch footprint of a count, keyed by (graph, anchor, |L|, |R|),
// remembered after the count first runs (serving admission).
struct FootKey {
    const void *graph;
    int anchor, k, kq;
    bool operator<(const FootKey &o) const {
        if (graph != o.graph) return graph < o.graph;
        if (anchor != o.anchor) return anchor < o.anchor;
        return k != o.k ? k < o.k : kq < o.kq;
    }
};

struct Server;

struct gbc_ctx_s {
    int device = 0;
    size_t budget = 0;
    int n_sms = 0;
    cudaStream_t own = nullptr;
    Lane lane;                               // the lane of the synchronous calls
    std::mutex tune_mu;
    std::map<TuneKey, int> tuned_anchor;     // filled by gbc_autotune
    std::map<TuneKey, int> tuned_warps;      // enumeration warps gbc_autotune measured faster than the default
    std::map<FootKey, size_t> footprint;     // exact scratch bytes of counts that ran (tune_mu)
    std::mutex mu;
    int live_graphs = 0;
    Server *server = nullptr;                // gbc_submit / gbc_poll
};

struct gbc_graph_s {
    gbc_ctx_s *ctx = nullptr;
    int32_t nU = 0, nV = 0;
    int64_t nE = 0;
    int32_t *offU = nullptr, *adjU = nullptr, *offV = nullptr, *adjV = nullptr;
    int32_t *degU = nullptr, *degV = nullptr;
    int32_t *adjV_byU = nullptr, *mirrorU = nullptr;  // anchor U: V rows by U rank, U-edge mirrors
    int32_t *adjU_byV = nullptr, *mirrorV = nullptr;  // anchor V
    int32_t maxdegU = 0, maxdegV = 0;
    unsigned long long wedgesU = 0, wedgesV = 0;      // sum C(deg, 2) on each side
    ulonglong2 *binom = nullptr;
    int32_t *n_ovf = nullptr;
    int32_t binom_nmax = 0;
    int32_t *callerU = nullptr, *callerV = nullptr;  // caller's id of every (renumbered) vertex
    std::vector<int32_t> callerU_h, callerV_h;
    // per anchor side (0: U, 1: V): sum omega, sum omega * row_stride(deg),
    // max omega, roots with omega > 0, sum omega^2 (double bits); omega(u) =
    // oriented wedges of root u.  They bound a count's scratch before it runs.
    unsigned long long fp[2][5] = {};
};

// Stream-ordered scratch that is released when the owner goes out of scope.
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    size_t bytes = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
    template <typename T>
    cudaError_t get(T **p, size_t n) {
        size_t b = std::max<size_t>(n, 1) * sizeof(T);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), b, st);
        if (e == cudaSuccess) { ptrs.push_back(*p); bytes += b; }
        return e;
    }
};

static void stop_server(gbc_ctx_s *ctx);

extern "C" {

const char *gbc_status_string(gbc_status s) {
    switch (s) {
        case GBC_OK: return "ok";
        case GBC_ERR_ARG: return "invalid argument";
        case GBC_ERR_INVALID_GRAPH: return "invalid graph";
        case GBC_ERR_OOM: return "out of device memory or budget";
        case GBC_ERR_OVERFLOW: return "count exceeds 2^128-1";
        case GBC_ERR_TIMEOUT: return "timeout";
        case GBC_ERR_CUDA: return "CUDA error";
        case GBC_PENDING: return "pending";
        case GBC_ERR_REJECTED: return "rejected";
    }
    return "unknown status";
}

const char *gbc_last_error(void) { return t_err; }

gbc_status gbc_ctx_create(int device, size_t mem_budget_bytes, gbc_ctx_t *out) {
    if (!out) return fail(GBC_ERR_ARG, "gbc_ctx_create: out is null");
    int n = 0;
    CK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(GBC_ERR_ARG, "gbc_ctx_create: device %d of %d", device, n);
    CK(cudaSetDevice(device));
    gbc_ctx_s *c = new gbc_ctx_s();
    c->device = device;
    CK(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device));
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.8 * (double)free_b);
    CK(init_enumerate_tables());
    CK(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
    CK(c->lane.create(c->own));
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return GBC_OK;
}

gbc_status gbc_ctx_set_stream(gbc_ctx_t ctx, void *stream) {
    if (!ctx) return fail(GBC_ERR_ARG, "gbc_ctx_set_stream: null context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->lane.st = stream ? reinterpret_cast<cudaStream_t>(stream) : ctx->own;
    return GBC_OK;
}

void gbc_ctx_destroy(gbc_ctx_t ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    stop_server(ctx);
    cudaStreamSynchronize(ctx->lane.st);
    ctx->lane.destroy();
    cudaStreamDestroy(ctx->own);
    delete ctx;
}

void gbc_free_graph(gbc_graph_t g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    cudaStream_t st = g->ctx->lane.st;
    void *ps[] = {g->offU, g->adjU, g->offV, g->adjV, g->degU, g->degV, g->adjV_byU,
                  g->mirrorU, g->adjU_byV, g->mirrorV, g->binom, g->n_ovf, g->callerU, g->callerV};
    for (void *p : ps)
        if (p) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    {
        std::lock_guard<std::mutex> lk(g->ctx->mu);
        g->ctx->live_graphs -= 1;
    }
    {
        std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
        for (auto it = g->ctx->tuned_anchor.begin(); it != g->ctx->tuned_anchor.end();)
            it = it->first.graph == g ? g->ctx->tuned_anchor.erase(it) : std::next(it);
        for (auto it = g->ctx->footprint.begin(); it != g->ctx->footprint.end();)
            it = it->first.graph == g ? g->ctx->footprint.erase(it) : std::next(it);
        for (auto it = g->ctx->tuned_warps.begin(); it != g->ctx->tuned_warps.end();)
            it = it->first.graph == g ? g->ctx->tuned_warps.erase(it) : std::next(it);
    }
    delete g;
}

gbc_status gbc_graph_info(gbc_graph_t g, int32_t *nU, int32_t *nV, int64_t *nE, int32_t *max_deg_u,
                          int32_t *max_deg_v) {
    if (!g) return fail(GBC_ERR_ARG, "gbc_graph_info: null graph");
    if (nU) *nU = g->nU;
    if (nV) *nV = g->nV;
    if (nE) *nE = g->nE;
    if (max_deg_u) *max_deg_u = g->maxdegU;
    if (max_deg_v) *max_deg_v = g->maxdegV;
    return GBC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// graph loading
// Renumbering at load time: each side by descending degree, ties in the
// caller's order.  Hubs' rows then sit together, which shortens the 2-hop
// expansion's reach through memory (the global-id reordering of Sec. V-B,
// Border, has the same aim; the bitmaps here are per root, so only locality
// is at stake).  Because ties keep the caller's order, the rank order
// (degree, id) of Def. 2 is unchanged and every search tree is the caller's.
// Two counting-sort passes build the renumbered CSRs with sorted rows: V rows
// by walking the new U order, then U rows by walking the new V order.
static void order_by_degree(int32_t n, const int32_t *off, std::vector<int32_t> &fresh, std::vector<int32_t> &caller) {
    int32_t maxd = 0;
    for (int32_t v = 0; v < n; ++v) maxd = std::max(maxd, off[v + 1] - off[v]);
    std::vector<int64_t> start((size_t)maxd + 1, 0);
    for (int32_t v = 0; v < n; ++v) start[off[v + 1] - off[v]] += 1;
    int64_t run = 0;
    for (int32_t d = maxd; d >= 0; --d) {
        const int64_t c = start[d];
        start[d] = run;
        run += c;
    }
    fresh.resize(n);
    caller.resize(n);
    for (int32_t v = 0; v < n; ++v) {
        const int32_t nv = (int32_t)start[off[v + 1] - off[v]]++;
        fresh[v] = nv;
        caller[nv] = v;
    }
}

static void renumber_by_degree(int32_t nU, int32_t nV, const int32_t *offU, const int32_t *adjU, const int32_t *offV,
                               std::vector<int32_t> &offU2, std::vector<int32_t> &adjU2, std::vector<int32_t> &offV2,
                               std::vector<int32_t> &adjV2, std::vector<int32_t> &callerU,
                               std::vector<int32_t> &callerV) {
    std::vector<int32_t> freshU, freshV;
    order_by_degree(nU, offU, freshU, callerU);
    order_by_degree(nV, offV, freshV, callerV);
    const int64_t E = offU[nU];
    offU2.assign((size_t)nU + 1, 0);
    offV2.assign((size_t)nV + 1, 0);
    adjU2.resize((size_t)E);
    adjV2.resize((size_t)E);
    for (int32_t v = 0; v < nV; ++v) offV2[v + 1] = offV2[v] + (offV[callerV[v] + 1] - offV[callerV[v]]);
    for (int32_t u = 0; u < nU; ++u) offU2[u + 1] = offU2[u] + (offU[callerU[u] + 1] - offU[callerU[u]]);
    std::vector<int32_t> cur(offV2.begin(), offV2.end() - 1);
    for (int32_t u = 0; u < nU; ++u) {
        const int32_t uo = callerU[u];
        for (int32_t e = offU[uo]; e < offU[uo + 1]; ++e) adjV2[cur[freshV[adjU[e]]]++] = u;
    }
    cur.assign(offU2.begin(), offU2.end() - 1);
    for (int32_t v = 0; v < nV; ++v)
        for (int32_t e = offV2[v]; e < offV2[v + 1]; ++e) adjU2[cur[adjV2[e]]++] = v;
}

static gbc_status load_common(gbc_ctx_t ctx, int32_t nU, int32_t nV, const int32_t *offU,
                              const int32_t *adjU, const int32_t *offV, const int32_t *adjV, bool host,
                              gbc_graph_t *out, int32_t flags = 0) {
    if (!ctx || !out || !offU || !offV) return fail(GBC_ERR_ARG, "gbc_load_graph: null argument");
    if (nU < 0 || nV < 0) return fail(GBC_ERR_ARG, "gbc_load_graph: negative vertex count");
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->lane.st;
    // |E| from the ends of the two offset arrays
    int32_t eU = 0, eV = 0;
    if (host) {
        eU = offU[nU];
        eV = offV[nV];
    } else {
        CK(cudaMemcpyAsync(&eU, offU + nU, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&eV, offV + nV, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (eU < 0 || eU != eV)
        return fail(GBC_ERR_INVALID_GRAPH, "gbc_load_graph: edge counts differ (U side %d, V side %d)", eU, eV);
    if (eU > 0 && (!adjU || !adjV)) return fail(GBC_ERR_ARG, "gbc_load_graph: null adjacency");
    gbc_graph_s *g = new gbc_graph_s();
    g->ctx = ctx;
    g->nU = nU;
    g->nV = nV;
    g->nE = eU;
    auto cleanup = [&](gbc_status s) {
        ctx->live_graphs += 1;  // gbc_free_graph decrements
        ctx->mu.unlock();
        gbc_free_graph(g);
        ctx->mu.lock();
        return s;
    };
#define CKG(expr)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return cleanup(fail(e_ == cudaErrorMemoryAllocation ? GBC_ERR_OOM : GBC_ERR_CUDA,      \
                                "%s: %s", #expr, cudaGetErrorString(e_)));                          \
    } while (0)
    const size_t E = (size_t)g->nE;
    CKG(cudaMallocAsync((void **)&g->offU, ((size_t)nU + 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->offV, ((size_t)nV + 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->adjU, std::max<size_t>(E, 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->adjV, std::max<size_t>(E, 1) * 4, st));
    const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CKG(cudaMemcpyAsync(g->offU, offU, ((size_t)nU + 1) * 4, kind, st));
    CKG(cudaMemcpyAsync(g->offV, offV, ((size_t)nV + 1) * 4, kind, st));
    if (E) {
        CKG(cudaMemcpyAsync(g->adjU, adjU, E * 4, kind, st));
        CKG(cudaMemcpyAsync(g->adjV, adjV, E * 4, kind, st));
    }
    // validation: offsets first, then rows and the transpose relation
    uint32_t *d_status = nullptr;
    int32_t *d_small = nullptr;               // maxdegU, maxdegV
    unsigned long long *d_wedges = nullptr;   // wedgesU, wedgesV
    CKG(cudaMallocAsync((void **)&d_status, 4, st));
    CKG(cudaMallocAsync((void **)&d_small, 8, st));
    CKG(cudaMallocAsync((void **)&d_wedges, 16, st));
    CKG(cudaMemsetAsync(d_status, 0, 4, st));
    CKG(cudaMemsetAsync(d_small, 0, 8, st));
    CKG(cudaMemsetAsync(d_wedges, 0, 16, st));
    uint32_t h_status = 0;
    CKG(launch_validate_offsets(g->offU, nU, g->nE, d_status, st));
    CKG(launch_validate_offsets(g->offV, nV, g->nE, d_status, st));
    CKG(cudaMemcpyAsync(&h_status, d_status, 4, cudaMemcpyDeviceToHost, st));
    CKG(cudaStreamSynchronize(st));
    if (h_status == 0) {
        CKG(launch_validate_rows(g->offU, g->adjU, nU, nV, d_status, st));
        CKG(launch_validate_rows(g->offV, g->adjV, nV, nU, d_status, st));
        CKG(cudaMemcpyAsync(&h_status, d_status, 4, cudaMemcpyDeviceToHost, st));
        CKG(cudaStreamSynchronize(st));
    }
    if (h_status == 0) {
        CKG(launch_validate_transpose(g->offU, g->adjU, nU, g->offV, g->adjV, d_status, st));
        CKG(cudaMemcpyAsync(&h_status, d_status, 4, cudaMemcpyDeviceToHost, st));
        CKG(cudaStreamSynchronize(st));
    }
    if (h_status != 0) {
        cudaFreeAsync(d_status, st);
        cudaFreeAsync(d_small, st);
        cudaFreeAsync(d_wedges, st);
        const char *why = (h_status & kStBadOffsets) ? "offsets not monotone or wrong ends"
                          : (h_status & kStBadRange) ? "neighbour id out of range"
                          : (h_status & kStUnsorted) ? "row not strictly increasing"
                                                     : "V-side CSR is not the transpose of the U side";
        return cleanup(fail(GBC_ERR_INVALID_GRAPH, "gbc_load_graph: %s", why));
    }
    // renumber both sides by degree (on the host) and replace the device copies
    if (flags & GBC_LOAD_KEEP_IDS) {
        g->callerU_h.resize((size_t)nU);
        g->callerV_h.resize((size_t)nV);
        for (int32_t u = 0; u < nU; ++u) g->callerU_h[u] = u;
        for (int32_t v = 0; v < nV; ++v) g->callerV_h[v] = v;
        CKG(cudaMallocAsync((void **)&g->callerU, std::max<size_t>(nU, 1) * 4, st));
        CKG(cudaMallocAsync((void **)&g->callerV, std::max<size_t>(nV, 1) * 4, st));
        if (nU) CKG(cudaMemcpyAsync(g->callerU, g->callerU_h.data(), (size_t)nU * 4, cudaMemcpyHostToDevice, st));
        if (nV) CKG(cudaMemcpyAsync(g->callerV, g->callerV_h.data(), (size_t)nV * 4, cudaMemcpyHostToDevice, st));
        CKG(cudaStreamSynchronize(st));
    } else {
        std::vector<int32_t> hoffU, hadjU, hoffV, hadjV;
        const int32_t *pOffU = offU, *pAdjU = adjU, *pOffV = offV;
        if (!host) {
            hoffU.resize((size_t)nU + 1);
            hoffV.resize((size_t)nV + 1);
            hadjU.resize(std::max<size_t>(E, 1));
            CKG(cudaMemcpyAsync(hoffU.data(), g->offU, ((size_t)nU + 1) * 4, cudaMemcpyDeviceToHost, st));
            CKG(cudaMemcpyAsync(hoffV.data(), g->offV, ((size_t)nV + 1) * 4, cudaMemcpyDeviceToHost, st));
            if (E) CKG(cudaMemcpyAsync(hadjU.data(), g->adjU, E * 4, cudaMemcpyDeviceToHost, st));
            CKG(cudaStreamSynchronize(st));
            pOffU = hoffU.data();
            pAdjU = hadjU.data();
            pOffV = hoffV.data();
        }
        std::vector<int32_t> offU2, adjU2, offV2, adjV2;
        renumber_by_degree(nU, nV, pOffU, pAdjU, pOffV, offU2, adjU2, offV2, adjV2, g->callerU_h, g->callerV_h);
        CKG(cudaMemcpyAsync(g->offU, offU2.data(), ((size_t)nU + 1) * 4, cudaMemcpyHostToDevice, st));
        CKG(cudaMemcpyAsync(g->offV, offV2.data(), ((size_t)nV + 1) * 4, cudaMemcpyHostToDevice, st));
        if (E) {
            CKG(cudaMemcpyAsync(g->adjU, adjU2.data(), E * 4, cudaMemcpyHostToDevice, st));
            CKG(cudaMemcpyAsync(g->adjV, adjV2.data(), E * 4, cudaMemcpyHostToDevice, st));
        }
        CKG(cudaMallocAsync((void **)&g->callerU, std::max<size_t>(nU, 1) * 4, st));
        CKG(cudaMallocAsync((void **)&g->callerV, std::max<size_t>(nV, 1) * 4, st));
        if (nU) CKG(cudaMemcpyAsync(g->callerU, g->callerU_h.data(), (size_t)nU * 4, cudaMemcpyHostToDevice, st));
        if (nV) CKG(cudaMemcpyAsync(g->callerV, g->callerV_h.data(), (size_t)nV * 4, cudaMemcpyHostToDevice, st));
        CKG(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    // degrees, per-side rank-sorted rows and mirror positions
    CKG(cudaMallocAsync((void **)&g->degU, std::max<size_t>(nU, 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->degV, std::max<size_t>(nV, 1) * 4, st));
    CKG(launch_degrees(g->offU, nU, g->degU, d_small, d_wedges, st));
    CKG(launch_degrees(g->offV, nV, g->degV, d_small + 1, d_wedges + 1, st));
    int32_t h_small[2];
    unsigned long long h_w[2];
    CKG(cudaMemcpyAsync(h_small, d_small, 8, cudaMemcpyDeviceToHost, st));
    CKG(cudaMemcpyAsync(h_w, d_wedges, 16, cudaMemcpyDeviceToHost, st));
    CKG(cudaStreamSynchronize(st));
    g->maxdegU = h_small[0];
    g->maxdegV = h_small[1];
    g->wedgesU = h_w[0];
    g->wedgesV = h_w[1];
    cudaFreeAsync(d_status, st);
    cudaFreeAsync(d_small, st);
    cudaFreeAsync(d_wedges, st);
    CKG(cudaMallocAsync((void **)&g->adjV_byU, std::max<size_t>(E, 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->adjU_byV, std::max<size_t>(E, 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->mirrorU, std::max<size_t>(E, 1) * 4, st));
    CKG(cudaMallocAsync((void **)&g->mirrorV, std::max<size_t>(E, 1) * 4, st));
    {
        int64_t *gtmp = nullptr;
        const int32_t maxrow = std::max(g->maxdegU, g->maxdegV);
        if (maxrow > 4096) {
            int64_t P = 1;
            while (P < maxrow) P <<= 1;
            CKG(cudaMallocAsync((void **)&gtmp, (size_t)P * 8 * 64, st));
        }
        // anchor U: V rows sorted by U rank; anchor V: U rows sorted by V rank
        CKG(launch_rank_sort_rows(g->offV, g->adjV, nV, g->degU, g->adjV_byU, g->maxdegV, gtmp, st));
        CKG(launch_rank_sort_rows(g->offU, g->adjU, nU, g->degV, g->adjU_byV, g->maxdegU, gtmp, st));
        if (gtmp) cudaFreeAsync(gtmp, st);
    }
    CKG(launch_mirror(g->offU, g->adjU, nU, g->offV, g->adjV_byU, g->degU, g->mirrorU, st));
    CKG(launch_mirror(g->offV, g->adjV, nV, g->offU, g->adjU_byV, g->degV, g->mirrorV, st));
    {
        unsigned long long *d_fp = nullptr;
        CKG(cudaMallocAsync((void **)&d_fp, sizeof(g->fp), st));
        CKG(cudaMemsetAsync(d_fp, 0, sizeof(g->fp), st));
        CKG(launch_footprint_sums(g->offU, nU, g->adjU, g->offV, g->mirrorU, d_fp, st));
        CKG(launch_footprint_sums(g->offV, nV, g->adjV, g->offU, g->mirrorV, d_fp + 5, st));
        CKG(cudaMemcpyAsync(g->fp, d_fp, sizeof(g->fp), cudaMemcpyDeviceToHost, st));
        CKG(cudaStreamSynchronize(st));
        cudaFreeAsync(d_fp, st);
    }
    // binomial table up to the largest degree (|C_R| never exceeds it)
    g->binom_nmax = std::max(std::max(g->maxdegU, g->maxdegV), 1);
    CKG(cudaMallocAsync((void **)&g->binom, (size_t)(g->binom_nmax + 1) * (kMaxPQ + 1) * sizeof(ulonglong2), st));
    CKG(cudaMallocAsync((void **)&g->n_ovf, (kMaxPQ + 1) * 4, st));
    CKG(launch_binomial(g->binom, g->n_ovf, g->binom_nmax, st));
    CKG(cudaStreamSynchronize(st));
#undef CKG
    ctx->live_graphs += 1;
    *out = g;
    return GBC_OK;
}

extern "C" gbc_status gbc_load_graph(gbc_ctx_t ctx, int32_t nU, int32_t nV, const int32_t *offU,
                                     const int32_t *adjU, const int32_t *offV, const int32_t *adjV,
                                     gbc_graph_t *out) {
    return load_common(ctx, nU, nV, offU, adjU, offV, adjV, true, out);
}

extern "C" gbc_status gbc_load_graph_ex(gbc_ctx_t ctx, int32_t nU, int32_t nV, const int32_t *offU,
                                        const int32_t *adjU, const int32_t *offV, const int32_t *adjV,
                                        int32_t flags, gbc_graph_t *out) {
    if (flags & ~GBC_LOAD_KEEP_IDS) return fail(GBC_ERR_ARG, "gbc_load_graph_ex: unknown flags 0x%x", flags);
    return load_common(ctx, nU, nV, offU, adjU, offV, adjV, true, out, flags);
}

extern "C" gbc_status gbc_load_graph_device(gbc_ctx_t ctx, int32_t nU, int32_t nV, const int32_t *offU_d,
                                            const int32_t *adjU_d, const int32_t *offV_d,
                                            const int32_t *adjV_d, gbc_graph_t *out) {
    return load_common(ctx, nU, nV, offU_d, adjU_d, offV_d, adjV_d, false, out);
}

// ---------------------------------------------------------------------------
// the count pipeline
static int pick_anchor(const gbc_graph_s *g, int p, int q) {
    // A side of size 1 needs no search at all; otherwise enumerate the smaller
    // set.  For p == q the cost has two regimes.  Up to p = q = 4 the 2-hop
    // candidate stage dominates: its wedges pass through the other side, so
    // anchor U costs sum_v C(deg v, 2) and anchor V sum_u C(deg u, 2); take the
    // cheaper.  From p = q = 5 on the deep subtrees dominate: anchor the side
    // with the lighter degree tail (smaller sum of C(deg, 2) over its own
    // vertices), whose roots have narrower C_R rows and sparser compatibility.
    if (p == 1) return GBC_ANCHOR_U;
    if (q == 1) return GBC_ANCHOR_V;
    if (p < q) return GBC_ANCHOR_U;
    if (q < p) return GBC_ANCHOR_V;
    if (p <= 4) return g->wedgesV <= g->wedgesU ? GBC_ANCHOR_U : GBC_ANCHOR_V;
    return g->wedgesU <= g->wedgesV ? GBC_ANCHOR_U : GBC_ANCHOR_V;
}

struct Timer {
    cudaEvent_t ev[5];
    bool on = false;
    void init(bool enable) {
        on = enable;
        if (on)
            for (auto &e : ev) cudaEventCreate(&e);
    }
    void mark(int i, cudaStream_t st) {
        if (on) cudaEventRecord(ev[i], st);
    }
    float between(int a, int b) {
        float ms = 0.f;
        if (on) cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return ms;
    }
    ~Timer() {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

// Small per-count device state: the u128 sum, status, tier sizes, work
// counters, totals of the per-root scans and the enumeration's word count.
struct Small {
    unsigned long long acc[2];
    int64_t totals[3];
    uint32_t status;
    int32_t tier_count[3];
    int32_t omega_max[3];
    int32_t queues[8];
    int32_t n_units;
    int32_t cand_max;
    unsigned long long deadline;
    unsigned long long enum_words;
    int32_t fin[2];   // completion counters (DoneRec publishing)
    unsigned long long tail[5];  // enumeration launch: start, last exit, exit sum (us), longest unit, warps
};

// One count of a (possibly one-element) batch.
struct Job {
    gbc_graph_s *g = nullptr;
    int p = 0, q = 0, anchor = 0;
    int time_limit_ms = 0;  // > 0: this job's own device deadline
    unsigned long long *per_root = nullptr;
    CountArgs a;
    Small h;
    bool trivial = false;
    size_t scratch_bytes = 0;  // device scratch held while this job ran
    size_t base_bytes = 0;     // scratch of the root classification and scans (before the waves)
    int pieces = 1;            // root ranges the count ran in (> 1: its scratch exceeded the budget)
    // listing mode (gbc_list_*): 1 sizes every root's records, 2 writes those
    // of roots [list_begin, list_end) (library ids) into list_out
    int list_mode = 0;
    int32_t list_begin = 0, list_end = 0;
    std::vector<int64_t> *list_sizes = nullptr;        // mode 1: 2 * |anchor side| (words, records)
    const std::vector<int64_t> *list_offsets = nullptr; // mode 2: per root of the range
    int32_t *list_out = nullptr;                        // mode 2: device buffer
    gbc_status st = GBC_OK;
    char err[256] = "";
    void set_error(gbc_status s, const char *fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, sizeof err, fmt, ap);
        va_end(ap);
        st = s;
    }
};

// Scratch bytes a count of (g, p, q) from `anchor` holds: the exact figure if
// the same count ran before on this context (*exact = 1), else an upper bound
// from the load-time wedge sums (*exact = 0).  Root u keeps at most
// c <= omega(u) / kq candidates (each needs kq wedges), with R rows of
// row_stride(d) words each; for |L| >= 4 its S and T blocks take
// (c + 32 row_stride(d)) ceil(c / 32) words, at most
// c^2 / 32 + 3c + c row_stride(d) + d + 64.
static size_t footprint_of(const gbc_graph_s *g, int anchor, int p, int q, int *exact) {
    const int k = anchor == GBC_ANCHOR_U ? p : q, kq = anchor == GBC_ANCHOR_U ? q : p;
    {
        std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
        auto it = g->ctx->footprint.find(FootKey{g, anchor, k, kq});
        if (it != g->ctx->footprint.end()) {
            if (exact) *exact = 1;
            return it->second;
        }
    }
    if (exact) *exact = 0;
    const int side = anchor == GBC_ANCHOR_U ? 0 : 1;
    const int64_t nA = side == 0 ? g->nU : g->nV;
    const unsigned long long *f = g->fp[side];
    double sq;
    memcpy(&sq, &f[4], sizeof sq);
    const double so = (double)f[0], sos = (double)f[1], omax = (double)f[2], npos = (double)f[3];
    double base = (double)sizeof(Small) + 20.0 * nA + 24.0 * (nA + 1) + 24.0 * ((nA + 1) / 2048 + 2);
    if (k >= 2 && omax > kCtaTierOmega) {  // global-table tier: one hash slab per CTA
        double slots = 32, sortcap = 1;
        while (slots < 2 * omax) slots *= 2;
        while (sortcap < omax) sortcap *= 2;
        base += 4.0 * (2 * slots + 2 * sortcap) * std::min(2.0 * g->ctx->n_sms, std::max(npos, 1.0));
    }
    if (k <= 2) return (size_t)base;
    const double c = so / kq, r = sos / kq;
    const double sw = k >= 4 ? sq / (32.0 * kq * (double)kq) + 3.0 * c + r + (double)g->nE + 64.0 * npos : 0.0;
    const double need = 12.0 * c + 4.0 * r + 4.0 * sw + 8.0 * (double)std::max<int64_t>(g->nE, 1) +
                        (k >= 4 ? 17.0 * c : 0.0);
    const double tot = base + need;
    return tot >= 1.8e19 ? (size_t)-1 : (size_t)tot;
}

// Outcome of job i of a batch, handed over as soon as it is known.
typedef std::function<void(int, gbc_status, gbc_u128, const char *)> DoneFn;

// Status of a job from its device status word (the job's own error first).
static gbc_status classify(const Job &J, uint32_t status, char *msg, size_t n) {
    if (J.st != GBC_OK) { snprintf(msg, n, "%s", J.err); return J.st; }
    if (status & kStTimeout) { snprintf(msg, n, "gbc_count: (%d,%d) passed its time limit", J.p, J.q); return GBC_ERR_TIMEOUT; }
    if (status & kStOverflow) { snprintf(msg, n, "gbc_count: (%d,%d) count exceeds 2^128-1", J.p, J.q); return GBC_ERR_OVERFLOW; }
    if (status) { snprintf(msg, n, "gbc_count: device status 0x%x", status); return GBC_ERR_CUDA; }
    msg[0] = 0;
    return GBC_OK;
}

// Scratch bytes of the wave phase of a job with |L| = k, from its per-root
// scan totals (candidates, R words, S words) and |E|: candidate ids and roots,
// per-edge position counts and maps, the R and S(+T) blocks, and for k >= 4
// the unit lists.
static size_t wave_need(int k, const int64_t totals[3], int64_t nE) {
    size_t b = (size_t)totals[0] * 8 + (size_t)std::max<int64_t>(totals[1], 1) * 4 +
               (size_t)std::max<int64_t>(nE, 1) * 8;
    if (k >= 4) b += (size_t)std::max<int64_t>(totals[2], 1) * 4 + (size_t)totals[0] * 17 + sizeof(CountArgs) + 256;
    return b;
}

// Runs every job of the batch phase by phase on the context's stream: one host
// synchronisation after the root classification, one after the per-root
// scans, and one at the end, whatever the number of jobs.  The enumeration of
// all jobs with |L| >= 4 is one persistent launch (a job table on the device).
// Per-job scratch is granted in waves that fit the context's budget.
// The enumeration launch sets its kernel's dynamic shared-memory limit to the
// launch's own size just before launching; counts on several host threads
// (serving workers) must not interleave those two steps, or one thread's
// smaller limit undercuts another thread's launch.
static std::mutex g_enum_launch_mu;

// on_done (optional): called for each job as soon as its outcome is known --
// jobs that end early (trivial, |L| <= 2, no candidates) at the host
// synchronisations, the others when their last kernel work is done, which the
// device reports through host-mapped completion records while the rest of the
// batch is still running.
// Returns a batch-level error (CUDA failure); per-job outcomes are in job.st.
static gbc_status run_jobs(gbc_ctx_s *ctx, Lane &lane, size_t budget, std::vector<Job> &jobs,
                           const gbc_count_options *opt, bool want_stats, Timer &tm, SearchStats *hs_out,
                           const DoneFn *on_done = nullptr) {
    cudaStream_t st = lane.st;
    const int n = (int)jobs.size();
    // statistics of the full traversal (1) or of the executed one (2); subtree collapse unless turned off
    const int enum_mode = want_stats ? (opt && opt->collect_stats == 2 ? 2 : 1) : 0;
    const int collapse = !opt || opt->collapse_skip == 0 ? kCollapseSkipDefault
                                                          : (opt->collapse_skip < 0 ? -1 : opt->collapse_skip);
    Scratch sc(st);
    Small *d_small = nullptr;
    CK(sc.get(&d_small, n));
    CK(cudaMemsetAsync(d_small, 0, sizeof(Small) * n, st));
    if (on_done) CK(lane.ensure_done(n));
    std::vector<char> released(n, 0);
    auto release = [&](int i, const unsigned long long *acc, uint32_t status) {
        if (!on_done || released[i]) return;
        released[i] = 1;
        char msg[256];
        const gbc_status s = classify(jobs[i], status, msg, sizeof msg);
        (*on_done)(i, s, gbc_u128{acc[0], acc[1]}, msg);
    };
    // Waits for the stream, handing over the jobs of `ids` whose completion
    // records the device has published meanwhile.
    auto wait_releasing = [&](const std::vector<int> &ids) -> cudaError_t {
        while (true) {
            const cudaError_t q = cudaStreamQuery(st);
            for (int i : ids) {
                if (released[i]) continue;
                DoneRec *d = lane.done_h + i;
                if (__atomic_load_n(&d->flag, __ATOMIC_ACQUIRE)) {
                    const volatile DoneRec *vd = d;
                    const unsigned long long acc[2] = {vd->acc[0], vd->acc[1]};
                    release(i, acc, vd->status);
                }
            }
            if (q != cudaErrorNotReady) return q;
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    };
    SearchStats *d_stats = nullptr;
    if (want_stats) {
        CK(sc.get(&d_stats, 1));
        CK(cudaMemsetAsync(d_stats, 0, sizeof(SearchStats), st));
    }
    std::vector<Small> hs(n);
    // Per-job launches of a batch go to the auxiliary streams so that the
    // kernels of small jobs overlap; fork/join keep them ordered against the
    // context's stream.  A single job stays on the context's stream.
    const bool multi = n > 1;
    auto fork = [&]() -> cudaError_t {
        if (!multi) return cudaSuccess;
        cudaError_t e = cudaEventRecord(lane.fork_ev, st);
        for (int i = 0; i < kAuxStreams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(lane.aux[i], lane.fork_ev, 0);
        return e;
    };
    auto join = [&]() -> cudaError_t {
        if (!multi) return cudaSuccess;
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kAuxStreams && e == cudaSuccess; ++i) {
            e = cudaEventRecord(lane.join_ev[i], lane.aux[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, lane.join_ev[i], 0);
        }
        return e;
    };
    auto sj = [&](int i) { return multi ? lane.aux[i % kAuxStreams] : st; };
    tm.mark(0, st);
    // ---- phase 0: arguments; single-vertex sets finish here
    for (int i = 0; i < n; ++i) {
        Job &J = jobs[i];
        gbc_graph_s *g = J.g;
        CountArgs &a = J.a;
        memset(&a, 0, sizeof a);
        if (J.anchor == GBC_ANCHOR_U) {
            a.g = SideView{g->nU, g->nV, g->offU, g->adjU, g->offV, g->adjV_byU, g->mirrorU, g->degU, g->maxdegU,
                           g->callerU};
            a.k = J.p;
            a.kq = J.q;
        } else {
            a.g = SideView{g->nV, g->nU, g->offV, g->adjV, g->offU, g->adjU_byV, g->mirrorV, g->degV, g->maxdegV,
                           g->callerV};
            a.k = J.q;
            a.kq = J.p;
        }
        a.binom = BinomTable{g->binom, g->n_ovf, g->binom_nmax};
        a.root_begin = 0;
        a.root_end = a.g.nA;
        a.lib_begin = 0;
        a.lib_end = a.g.nA;
        a.cand_base = 0;
        a.position_order = opt ? opt->position_order : 0;
        if (opt && opt->root_end > opt->root_begin) {
            a.root_begin = std::max(0, opt->root_begin);
            a.root_end = std::min(a.g.nA, opt->root_end);
        }
        Small *s = d_small + i;
        a.fin = s->fin;
        a.done = on_done ? lane.done_d + i : nullptr;
        a.acc = s->acc;
        a.status = &s->status;
        a.tier_count = s->tier_count;
        a.omega_max = s->omega_max;
        a.queues = s->queues;
        a.n_units = &s->n_units;
        a.cand_max = &s->cand_max;
        a.deadline = &s->deadline;
        a.enum_words = &s->enum_words;
        a.tail = s->tail;
        a.stats = d_stats;
        a.per_root = J.per_root;
        J.trivial = (a.k > a.g.nA) || (a.kq > a.g.maxdegA) || a.g.nA == 0;
        if (!J.trivial && a.k == 1) CK(launch_single_vertex_sets(a, st));
    }
    for (int i = 0; i < n; ++i) {
        const int lim = jobs[i].time_limit_ms > 0 ? jobs[i].time_limit_ms : (opt ? opt->time_limit_ms : 0);
        if (lim > 0) CK(launch_set_deadline(&d_small[i].deadline, (unsigned long long)lim * 1000000ull, st));
    }
    auto active = [&](const Job &J) { return J.st == GBC_OK && !J.trivial && J.a.k >= 2; };
    // ---- phase 1: oriented wedge counts and root tiers
    bool any = false;
    for (Job &J : jobs) {
        if (!active(J)) continue;
        const int64_t nA = J.a.g.nA;
        const size_t b0 = sc.bytes;
        CK(sc.get(&J.a.omega, nA));
        CK(sc.get(&J.a.tier_list, 3 * nA));
        CK(sc.get(&J.a.cand_count, nA));
        J.base_bytes += sc.bytes - b0 + sizeof(Small);
        any = true;
    }
    CK(fork());
    for (int i = 0; i < n; ++i)
        if (active(jobs[i])) CK(launch_root_omega(jobs[i].a, sj(i)));
    CK(join());
    if (any) {
        CK(cudaMemcpyAsync(hs.data(), d_small, sizeof(Small) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i)  // trivial and single-vertex jobs are complete
            if (!active(jobs[i])) release(i, hs[i].acc, hs[i].status);
    }
    // ---- phase 2: candidates (pass A) and, for |L| >= 3, the per-root offsets
    any = false;
    std::vector<int64_t *> scan_tmp(n, nullptr);
    for (int i = 0; i < n; ++i) {
        Job &J = jobs[i];
        if (!active(J)) continue;
        CountArgs &a = J.a;
        const Small &h = hs[i];
        const size_t b0 = sc.bytes;
        if (h.tier_count[2] > 0) {
            if (h.omega_max[2] > (1 << 28)) {
                J.set_error(GBC_ERR_OOM, "gbc_count: a root has %d oriented wedges (limit 2^28)", h.omega_max[2]);
                continue;
            }
            int64_t slots = 32, sortcap = 1;
            while (slots < 2 * (int64_t)h.omega_max[2]) slots <<= 1;
            while (sortcap < h.omega_max[2]) sortcap <<= 1;
            a.slab_words = 2 * slots + 2 * sortcap;
            // one slab per CTA of the global-table tier, as many CTAs as fit in a
            // quarter of the context's budget (at least one): a root's table must
            // fit whole (the exact footprints that serving reserves include them)
            const size_t slab_bytes = (size_t)a.slab_words * 4;
            const int64_t fit = (int64_t)(ctx->budget / 4 / slab_bytes);
            if (fit < 1) {
                J.set_error(GBC_ERR_OOM, "gbc_count: a root's wedge table (%zu B) exceeds a quarter of the budget",
                            slab_bytes);
                continue;
            }
            a.slab_ctas = (int32_t)std::min<int64_t>(std::min(ctx->n_sms * 2, h.tier_count[2]), fit);
            CK(sc.get(&a.slab, (size_t)a.slab_words * a.slab_ctas));
        }
        if (a.k >= 3 || J.list_mode) {
            const int64_t nA = a.g.nA;
            int64_t *cand_off, *r_off, *s_off;
            CK(sc.get(&cand_off, nA + 1));
            CK(sc.get(&r_off, nA + 1));
            CK(sc.get(&s_off, nA + 1));
            CK(sc.get(&scan_tmp[i], 3 * ((nA + 1) / 2048 + 2)));
            a.cand_off = cand_off;
            a.r_off = r_off;
            a.s_off = s_off;
            any = true;
        }
        J.base_bytes += sc.bytes - b0;
    }
    CK(fork());
    for (int i = 0; i < n; ++i) {
        Job &J = jobs[i];
        if (!active(J)) continue;
        CountArgs &a = J.a;
        CK(launch_candidates(a, false, hs[i].tier_count, ctx->n_sms, sj(i)));
        if (a.k >= 3 || J.list_mode)
            CK(launch_root_offsets(a, const_cast<int64_t *>(a.cand_off), const_cast<int64_t *>(a.r_off),
                                   const_cast<int64_t *>(a.s_off), scan_tmp[i], d_small[i].totals, sj(i)));
    }
    CK(join());
    tm.mark(1, st);
    const bool sized = any;  // the scan totals of every |L| >= 3 job are on the host
    if (any) {
        CK(cudaMemcpyAsync(hs.data(), d_small, sizeof(Small) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    // ---- phase 3 (in waves): bitmap rows, pairwise rows, enumeration
    std::vector<int> todo;
    for (int i = 0; i < n; ++i) {
        Job &J = jobs[i];
        if (!active(J) || J.a.k < 3 || J.list_mode) continue;
        J.a.n_cand = hs[i].totals[0];
        if (J.a.n_cand == 0) continue;
        if (J.a.n_cand >= INT32_MAX) {
            J.set_error(GBC_ERR_OOM, "gbc_count: %lld candidates exceed one launch", (long long)J.a.n_cand);
            continue;
        }
        todo.push_back(i);
    }
    auto need_of = [&](int i) { return wave_need(jobs[i].a.k, hs[i].totals, jobs[i].g->nE); };
    const bool csr = opt && opt->kernel == GBC_KERNEL_CSR;
    // enumeration warps of a launch over `ids`: the option, else the tuned warps
    // of its jobs when every one of them has some (their largest), else 0 (auto)
    auto warps_for = [&](const std::vector<int> &ids) -> int {
        if (opt && opt->enum_warps > 0) return opt->enum_warps;
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        int w = 0;
        for (int i : ids) {
            if (jobs[i].a.k < 4) continue;
            auto it = ctx->tuned_warps.find(TuneKey{jobs[i].g, jobs[i].p, jobs[i].q});
            if (it == ctx->tuned_warps.end()) return 0;
            w = std::max(w, it->second);
        }
        return w;
    };
    std::vector<char> in_todo(n, 0);
    for (int i : todo) in_todo[i] = 1;
    // exact footprint of each job that got through the scans (serving admission)
    std::vector<size_t> foot(n, 0);
    for (int i = 0; i < n; ++i)
        if (active(jobs[i]) && jobs[i].st == GBC_OK) foot[i] = jobs[i].base_bytes + (in_todo[i] ? need_of(i) : 0);
    if (sized) {
        // everything not waiting for the waves is complete (|L| = 2 summed its
        // leaves in pass A; no candidates means a zero count)
        for (int i = 0; i < n; ++i)
            if (!in_todo[i]) release(i, hs[i].acc, hs[i].status);
    }
    // A job whose search scratch exceeds the budget on its own runs in pieces:
    // contiguous ranges of roots (library ids), cut where the exact per-root
    // scratch (from the scans' offsets) reaches the budget, one after the
    // other.  Roots' search trees are independent, so the pieces need nothing
    // from each other and add into the job's sum (the closure partitioning of
    // Sec. VI, applied to the scratch; the graph itself stays resident).
    auto run_in_pieces = [&](int i, size_t avail) -> gbc_status {
        Job &J = jobs[i];
        if (opt && opt->kernel == GBC_KERNEL_CSR) {
            J.set_error(GBC_ERR_OOM, "gbc_count: the sorted-list ablation runs whole; its scratch exceeds the budget");
            return GBC_OK;
        }
        const CountArgs &a = J.a;
        const int64_t nA = a.g.nA;
        const bool k4 = a.k >= 4;
        std::vector<int64_t> co((size_t)nA + 1), ro((size_t)nA + 1), so((size_t)nA + 1);
        CK(cudaMemcpyAsync(co.data(), a.cand_off, (size_t)(nA + 1) * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ro.data(), a.r_off, (size_t)(nA + 1) * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(so.data(), a.s_off, (size_t)(nA + 1) * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        auto pre = [&](int64_t u) -> size_t {
            return (size_t)co[u] * 8 + (size_t)ro[u] * 4 + (k4 ? (size_t)so[u] * 4 + (size_t)co[u] * 17 : 0);
        };
        const int64_t nE = std::max<int64_t>(J.g->nE, 1);
        const size_t fixed = (size_t)nE * 8 + (k4 ? sizeof(CountArgs) + 256 : 0) + 4096;
        if (avail <= fixed) {
            J.set_error(GBC_ERR_OOM, "gbc_count: budget %zu B below the %zu B a count of this graph needs", avail, fixed);
            return GBC_OK;
        }
        const size_t room = avail - fixed;
        std::vector<std::pair<int64_t, int64_t>> pieces;
        for (int64_t lb = 0; lb < nA;) {
            int64_t lo = lb, hi = nA;  // the largest end with the range's scratch within room
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) / 2;
                if (pre(mid) - pre(lb) <= room) lo = mid;
                else hi = mid - 1;
            }
            if (lo == lb) {
                J.set_error(GBC_ERR_OOM, "gbc_count: one root needs %zu B of search scratch, more than the %zu B left",
                            pre(lb + 1) - pre(lb), room);
                return GBC_OK;
            }
            pieces.push_back({lb, lo});
            lb = lo;
        }
        J.pieces = (int)pieces.size();
        for (const auto &pc : pieces) {
            const int64_t pb = pc.first, pe = pc.second, nc = co[pe] - co[pb];
            if (nc == 0) continue;
            Scratch psc(st);
            CountArgs b = a;
            b.lib_begin = (int32_t)pb;
            b.lib_end = (int32_t)pe;
            b.cand_base = co[pb];
            b.n_cand = nc;
            b.done = nullptr;  // released when the last piece is done
            int32_t *cand_p = nullptr, *root_p = nullptr;
            uint32_t *R_p = nullptr, *S_p = nullptr;
            CK(psc.get(&b.poscnt, nE));
            CK(psc.get(&b.posmap, nE));
            CK(cudaMemsetAsync(b.poscnt, 0, (size_t)nE * 4, st));
            CK(psc.get(&cand_p, nc));
            CK(psc.get(&root_p, nc));
            CK(psc.get(&R_p, ro[pe] - ro[pb]));
            CK(cudaMemsetAsync(R_p, 0, (size_t)std::max<int64_t>(ro[pe] - ro[pb], 1) * 4, st));
            // global offsets of the piece's roots land in its own buffers
            b.cand = cand_p - co[pb];
            b.cand_root = root_p - co[pb];
            b.R = R_p - ro[pb];
            int2 *u_all = nullptr, *u_sorted = nullptr;
            uint8_t *u_bucket = nullptr;
            int32_t *ucnt = nullptr;
            if (k4) {
                CK(psc.get(&S_p, so[pe] - so[pb]));
                CK(cudaMemsetAsync(S_p, 0, (size_t)std::max<int64_t>(so[pe] - so[pb], 1) * 4, st));
                b.S = S_p - so[pb];
                CK(psc.get(&u_all, nc));
                CK(psc.get(&u_sorted, nc));
                CK(psc.get(&u_bucket, nc));
                CK(psc.get(&ucnt, 33));
                CK(cudaMemsetAsync(ucnt, 0, 33 * 4, st));
                b.units_all = u_all;
                b.units_bucket = u_bucket;
                b.n_units_all = ucnt;
                b.bucket_count = ucnt + 1;
                b.job_id = 0;
            }
            // the pass-B and pairwise work counters start again for every piece
            CK(cudaMemsetAsync(&d_small[i].queues[3], 0, 5 * sizeof(int32_t), st));
            CK(launch_candidates(b, true, hs[i].tier_count, ctx->n_sms, st));
            CK(launch_pairs(b, ctx->n_sms, st));
            if (k4) {
                CountArgs *d_job = nullptr;
                int32_t *d_queue = nullptr;
                CK(psc.get(&d_job, 1));
                CK(psc.get(&d_queue, 1));
                CK(cudaMemsetAsync(d_queue, 0, 4, st));
                CK(cudaMemcpyAsync(d_job, &b, sizeof(CountArgs), cudaMemcpyHostToDevice, st));
                CK(launch_sort_units(u_all, u_bucket, ucnt, ucnt + 1, ucnt + 17, u_sorted, nc, st));
                {
                    std::lock_guard<std::mutex> lk(g_enum_launch_mu);
                    CK(launch_enumerate(d_job, u_sorted, ucnt, d_queue, enum_mode, collapse,
                                        warps_for(std::vector<int>{i}), (int)row_stride(a.g.maxdegA),
                                        (std::max(hs[i].cand_max, 1) + 31) / 32, a.k, ctx->n_sms, st));
                }
            }
            CK(cudaStreamSynchronize(st));  // b is read by the launch
            J.scratch_bytes = std::max(J.scratch_bytes, sc.bytes + psc.bytes);
        }
        return GBC_OK;
    };
    // Listing: pass B rows for the range's roots, then the listing kernel.
    auto run_listing = [&](int i) -> gbc_status {
        Job &J = jobs[i];
        CountArgs b = J.a;
        const int64_t nA = b.g.nA;
        const int32_t lb = J.list_begin, le = J.list_end;
        Scratch lsc(st);
        ListArgs L;
        memset(&L, 0, sizeof L);
        L.mode = J.list_mode;
        L.begin = lb;
        L.end = le;
        L.callerO = J.anchor == GBC_ANCHOR_U ? J.g->callerV : J.g->callerU;
        CK(lsc.get(&L.queue, 1));
        CK(cudaMemsetAsync(L.queue, 0, 4, st));
        if (L.mode == 1) {
            CK(lsc.get(&L.sizes, 2 * std::max<int64_t>(nA, 1)));
            CK(cudaMemsetAsync(L.sizes, 0, 16 * (size_t)std::max<int64_t>(nA, 1), st));
        } else {
            int64_t *offs = nullptr;
            CK(lsc.get(&offs, std::max<int32_t>(le - lb, 1)));
            if (le > lb)
                CK(cudaMemcpyAsync(offs, J.list_offsets->data(), 8 * (size_t)(le - lb), cudaMemcpyHostToDevice, st));
            L.offsets = offs;
            L.out = J.list_out;
        }
        const int64_t range = le - lb;
        int warps = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->n_sms * 32, range));
        bool launch = range > 0;
        if (b.k >= 2 && launch) {
            if (!active(J)) launch = false;  // nothing to list (p > |anchor| or q > max degree)
        }
        if (b.k >= 2 && launch) {
            int64_t ends[4];
            CK(cudaMemcpyAsync(&ends[0], b.cand_off + lb, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&ends[1], b.cand_off + le, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&ends[2], b.r_off + lb, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&ends[3], b.r_off + le, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            const int64_t nc = ends[1] - ends[0];
            const int64_t nE = std::max<int64_t>(J.g->nE, 1);
            int32_t *cand_p = nullptr, *root_p = nullptr;
            uint32_t *R_p = nullptr;
            CK(lsc.get(&b.poscnt, nE));
            CK(lsc.get(&b.posmap, nE));
            CK(cudaMemsetAsync(b.poscnt, 0, (size_t)nE * 4, st));
            CK(lsc.get(&cand_p, nc));
            CK(lsc.get(&root_p, nc));
            CK(lsc.get(&R_p, ends[3] - ends[2]));
            CK(cudaMemsetAsync(R_p, 0, (size_t)std::max<int64_t>(ends[3] - ends[2], 1) * 4, st));
            b.lib_begin = lb;
            b.lib_end = le;
            b.cand_base = ends[0];
            b.n_cand = nc;
            b.cand = cand_p - ends[0];
            b.cand_root = root_p - ends[0];
            b.R = R_p - ends[2];
            b.S = nullptr;
            b.done = nullptr;
            CK(cudaMemsetAsync(&d_small[i].queues[3], 0, 5 * sizeof(int32_t), st));
            if (nc > 0) CK(launch_candidates(b, true, hs[i].tier_count, ctx->n_sms, st));
            else launch = false;
            if (launch) {
                L.stack_words = list_stack_words(b.k, b.g.maxdegA, hs[i].cand_max);
                warps = (int)std::max<int64_t>(1, std::min<int64_t>(warps, (int64_t(1) << 28) / L.stack_words));
                CK(lsc.get(&L.stack, (size_t)warps * L.stack_words));
            }
        }
        if (launch) CK(launch_list(b, L, warps, st));
        if (L.mode == 1) {
            J.list_sizes->assign(2 * (size_t)nA, 0);
            if (nA > 0)
                CK(cudaMemcpyAsync(J.list_sizes->data(), L.sizes, 16 * (size_t)nA, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        J.scratch_bytes = std::max(J.scratch_bytes, sc.bytes + lsc.bytes);
        return GBC_OK;
    };
    for (int i = 0; i < n; ++i)
        if (jobs[i].list_mode && jobs[i].st == GBC_OK) {
            const gbc_status e = run_listing(i);
            if (e != GBC_OK) return e;
        }
    size_t pos = 0;
    while (pos < todo.size()) {
        Scratch wave_sc(st);
        std::vector<int> wave;
        size_t used = sc.bytes;
        for (; pos < todo.size(); ++pos) {
            const int i = todo[pos];
            const size_t need = need_of(i);
            if (used + need > budget) {
                if (wave.empty()) {
                    const gbc_status e = run_in_pieces(i, budget > used ? budget - used : 0);
                    if (e != GBC_OK) return e;
                    if (jobs[i].st != GBC_OK) {
                        const unsigned long long zero[2] = {0, 0};
                        release(i, zero, 0);
                    }
                    continue;
                }
                break;
            }
            used += need;
            wave.push_back(i);
        }
        // The wave's enumeration runs one persistent launch per |L| on the anchor
        // side: each launch's shared-memory layout (levels, row widths) is the
        // largest of its own counts', so a deep count's layout does not lower
        // the occupancy of the others.  Counts with the same |L| share a launch.
        struct EnumGroup {
            int k = 0;
            std::vector<CountArgs> jobs;
            int max_wr = 2, max_wl = 2;
            int64_t unit_cap = 0;
            int2 *units_all = nullptr, *units_sorted = nullptr;
            uint8_t *units_bucket = nullptr;
            int32_t *ucounters = nullptr;  // n_all, bucket_count[16], cursor[16]
            std::vector<int> ids;
        };
        std::vector<EnumGroup> groups;
        auto group_of = [&](int k) -> EnumGroup & {
            for (EnumGroup &G : groups)
                if (G.k == k) return G;
            groups.emplace_back();
            groups.back().k = k;
            return groups.back();
        };
        for (int i : wave)
            if (jobs[i].a.k >= 4) group_of(jobs[i].a.k).unit_cap += jobs[i].a.n_cand;
        std::sort(groups.begin(), groups.end(), [](const EnumGroup &x, const EnumGroup &y) { return x.k > y.k; });
        for (EnumGroup &G : groups) {
            if (G.unit_cap <= 0) continue;
            CK(wave_sc.get(&G.units_all, G.unit_cap));
            CK(wave_sc.get(&G.units_sorted, G.unit_cap));
            CK(wave_sc.get(&G.units_bucket, G.unit_cap));
            CK(wave_sc.get(&G.ucounters, 33));
            CK(cudaMemsetAsync(G.ucounters, 0, 33 * 4, st));
        }
        for (int i : wave) {
            CountArgs &a = jobs[i].a;
            const Small &h = hs[i];
            const int64_t nE = std::max<int64_t>(jobs[i].g->nE, 1);
            CK(wave_sc.get(&a.poscnt, nE));
            CK(wave_sc.get(&a.posmap, nE));
            CK(cudaMemsetAsync(a.poscnt, 0, (size_t)nE * 4, st));
            CK(wave_sc.get(&a.cand, a.n_cand));
            CK(wave_sc.get(&a.cand_root, a.n_cand));
            CK(wave_sc.get(&a.R, h.totals[1]));
            CK(cudaMemsetAsync(a.R, 0, std::max<int64_t>(h.totals[1], 1) * 4, st));
            if (a.k >= 4) {
                CK(wave_sc.get(&a.S, h.totals[2]));
                CK(cudaMemsetAsync(a.S, 0, std::max<int64_t>(h.totals[2], 1) * 4, st));
                EnumGroup &G = group_of(a.k);
                a.units_all = G.units_all;
                a.units_bucket = G.units_bucket;
                a.n_units_all = G.ucounters;
                a.bucket_count = G.ucounters + 1;
            }
        }
        CK(fork());
        for (int i : wave) CK(launch_candidates(jobs[i].a, true, hs[i].tier_count, ctx->n_sms, sj(i)));
        tm.mark(1, st);
        for (int i : wave) {
            CountArgs &a = jobs[i].a;
            const Small &h = hs[i];
            if (a.k >= 4) a.job_id = (int32_t)group_of(a.k).jobs.size();
            if (csr) continue;
            CK(launch_pairs(a, ctx->n_sms, sj(i)));
            if (a.k >= 4) {
                EnumGroup &G = group_of(a.k);
                G.jobs.push_back(a);
                G.ids.push_back(i);
                G.max_wr = std::max(G.max_wr, (int)row_stride(a.g.maxdegA));
                G.max_wl = std::max(G.max_wl, (std::max(h.cand_max, 1) + 31) / 32);
            }
        }
        CK(join());
        tm.mark(2, st);
        if (csr) {
            // the sorted-list ablation walks the same trees from pass B's candidate lists
            for (int i : wave) {
                CountArgs &a = jobs[i].a;
                CsrArgs C;
                memset(&C, 0, sizeof C);
                C.dmax = std::max(a.g.maxdegA, 1);
                C.cmax = std::max(hs[i].cand_max, 1);
                C.stack_words = csr_stack_words(a.k, C.dmax, C.cmax);
                const int warps = (int)std::max<int64_t>(
                    1, std::min<int64_t>((int64_t)ctx->n_sms * 32, (int64_t(1) << 28) / C.stack_words));
                CK(wave_sc.get(&C.queue, 1));
                CK(cudaMemsetAsync(C.queue, 0, 4, st));
                CK(wave_sc.get(&C.stack, (size_t)warps * C.stack_words));
                CK(launch_enumerate_csr(a, C, warps, want_stats, st));
            }
            CK(cudaStreamSynchronize(st));
            for (EnumGroup &G : groups) G.jobs.clear();
        }
        bool launched = false;
        for (EnumGroup &G : groups) {
            if (G.jobs.empty()) continue;
            CountArgs *d_jobs = nullptr;
            int32_t *d_queue = nullptr;
            CK(wave_sc.get(&d_jobs, G.jobs.size()));
            CK(wave_sc.get(&d_queue, 1));
            CK(cudaMemsetAsync(d_queue, 0, 4, st));
            CK(cudaMemcpyAsync(d_jobs, G.jobs.data(), sizeof(CountArgs) * G.jobs.size(),
                               cudaMemcpyHostToDevice, st));
            CK(launch_sort_units(G.units_all, G.units_bucket, G.ucounters, G.ucounters + 1, G.ucounters + 17,
                                 G.units_sorted, G.unit_cap, st));
            {
                std::lock_guard<std::mutex> lk(g_enum_launch_mu);
                CK(launch_enumerate(d_jobs, G.units_sorted, G.ucounters, d_queue, enum_mode, collapse,
                                    warps_for(G.ids), G.max_wr, G.max_wl, G.k, ctx->n_sms, st));
            }
            launched = true;
        }
        if (launched) {
            // the job tables are read by the launches: keep the host copies alive until they have run
            if (on_done) CK(wait_releasing(wave));
            else CK(cudaStreamSynchronize(st));
        } else if (on_done) {
            CK(wait_releasing(wave));  // |L| = 3 counts publish from the pairwise kernel
        }
        for (int i : wave) jobs[i].scratch_bytes = sc.bytes + wave_sc.bytes;
    }
    for (Job &J : jobs)
        if (J.scratch_bytes == 0) J.scratch_bytes = sc.bytes;
    tm.mark(3, st);
    CK(cudaMemcpyAsync(hs.data(), d_small, sizeof(Small) * n, cudaMemcpyDeviceToHost, st));
    if (d_stats && hs_out) CK(cudaMemcpyAsync(hs_out, d_stats, sizeof(SearchStats), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (!(opt && opt->root_end > opt->root_begin)) {  // remember full counts' footprints
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        for (int i = 0; i < n; ++i)
            if (foot[i]) ctx->footprint[FootKey{jobs[i].g, jobs[i].anchor, jobs[i].a.k, jobs[i].a.kq}] = foot[i];
    }
    for (int i = 0; i < n; ++i) {
        Job &J = jobs[i];
        J.h = hs[i];
        release(i, J.h.acc, J.h.status);
        if (J.st != GBC_OK) continue;
        char msg[256];
        const gbc_status s = classify(J, J.h.status, msg, sizeof msg);
        if (s != GBC_OK) J.set_error(s, "%s", msg);
    }
    return GBC_OK;
}

static int resolve_anchor(const gbc_graph_s *g, int p, int q, int requested) {
    if (requested) return requested;
    std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
    auto it = g->ctx->tuned_anchor.find(TuneKey{g, p, q});
    return it != g->ctx->tuned_anchor.end() ? it->second : pick_anchor(g, p, q);
}

static gbc_status count_impl(gbc_graph_t g, int p, int q, const gbc_count_options *opt, gbc_u128 *out,
                             gbc_count_info *info, int force_anchor, unsigned long long *per_root_dev) {
    if (!g || (!out && !per_root_dev)) return fail(GBC_ERR_ARG, "gbc_count: null argument");
    if (p < 1 || q < 1 || p > GBC_MAX_PQ || q > GBC_MAX_PQ)
        return fail(GBC_ERR_ARG, "gbc_count: p=%d q=%d outside [1, %d]", p, q, GBC_MAX_PQ);
    gbc_ctx_s *ctx = g->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    const int anchor = resolve_anchor(g, p, q, force_anchor ? force_anchor : (opt ? opt->anchor : 0));
    if (anchor != GBC_ANCHOR_U && anchor != GBC_ANCHOR_V) return fail(GBC_ERR_ARG, "gbc_count: bad anchor %d", anchor);
    if (opt && (opt->kernel < GBC_KERNEL_BITMAP || opt->kernel > GBC_KERNEL_CSR))
        return fail(GBC_ERR_ARG, "gbc_count: bad kernel %d", opt->kernel);
    const bool want_stats = opt && opt->collect_stats;
    std::vector<Job> jobs(1);
    jobs[0].g = g;
    jobs[0].p = p;
    jobs[0].q = q;
    jobs[0].anchor = anchor;
    jobs[0].per_root = per_root_dev;
    t_launches = 0;
    Timer tm;
    tm.init(info != nullptr);
    SearchStats hs;
    memset(&hs, 0, sizeof hs);
    gbc_status s = run_jobs(ctx, ctx->lane, ctx->budget, jobs, opt, want_stats, tm, &hs);
    if (s != GBC_OK) return s;
    Job &J = jobs[0];
    if (J.st != GBC_OK) return fail(J.st, "%s", J.err);
    if (info) {
        gbc_count_info inf;
        memset(&inf, 0, sizeof inf);
        inf.anchor_used = anchor;
        inf.set_size = J.a.k;
        inf.roots = (int64_t)hs.roots;
        inf.candidates = J.h.totals[0] ? J.h.totals[0] : (int64_t)hs.cands;
        inf.units = want_stats ? (int64_t)hs.units : J.h.n_units;
        for (int l = 0; l <= GBC_MAX_PQ; ++l) {
            inf.evals[l] = (int64_t)hs.evals[l];
            inf.passed[l] = (int64_t)hs.passed[l];
        }
        inf.words_r = (int64_t)hs.words_r;
        inf.words_l = (int64_t)hs.words_l;
        inf.words_enum = (int64_t)hs.words_enum;
        inf.words_exec = (int64_t)hs.words_exec;
        inf.collapsed = (int64_t)hs.collapsed;
        for (int i = 0; i < 10; ++i) inf.enum_phase_cycles[i] = (int64_t)hs.phase_cycles[i];
        inf.scratch_bytes = (int64_t)J.scratch_bytes;
        if (!J.trivial && J.a.k >= 2) {
            inf.ms_candidates = tm.between(0, 1);
            if (J.a.k >= 3 && J.a.n_cand > 0) {
                inf.ms_pairs = tm.between(1, 2);
                inf.ms_enumerate = J.a.k >= 4 ? tm.between(2, 3) : 0.f;
            }
        }
        inf.ms_total = tm.between(0, 3);
        inf.enum_words = (int64_t)J.h.enum_words;
        inf.launches = t_launches;
        inf.pieces = J.pieces;
        {
            // the enumeration launch's longest unit and how long before its end its
            // warps left on average (every warp of the launch times its own exit)
            const unsigned long long *tl = J.h.tail;
            inf.enum_longest_unit_ms = (float)((double)tl[3] / 1e6);
            if (tl[0] && tl[1] > tl[0] && tl[4] > 0) {
                const double span_ms = ((double)tl[1] - (double)tl[0]) / 1e6;
                const double mean_exit_ms = (double)tl[2] / 1e3 / (double)tl[4];
                inf.enum_span_ms = (float)span_ms;
                inf.enum_exit_spread_ms = (float)(span_ms - mean_exit_ms);
            }
        }
        *info = inf;
    }
    if (out) {
        out->lo = J.h.acc[0];
        out->hi = J.h.acc[1];
    }
    return GBC_OK;
}

extern "C" gbc_status gbc_count_batch(gbc_ctx_t ctx, int n, const gbc_graph_t *graphs, const int *p,
                                      const int *q, gbc_u128 *out, gbc_status *per_job) {
    if (!ctx || n < 0 || (n > 0 && (!graphs || !p || !q || !out || !per_job)))
        return fail(GBC_ERR_ARG, "gbc_count_batch: null argument");
    if (n == 0) return GBC_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<Job> jobs;
    std::vector<int> slot;
    jobs.reserve(n);
    for (int i = 0; i < n; ++i) {
        per_job[i] = GBC_OK;
        out[i] = gbc_u128{0, 0};
        if (!graphs[i] || graphs[i]->ctx != ctx) { per_job[i] = GBC_ERR_ARG; continue; }
        if (p[i] < 1 || q[i] < 1 || p[i] > GBC_MAX_PQ || q[i] > GBC_MAX_PQ) { per_job[i] = GBC_ERR_ARG; continue; }
        Job J;
        J.g = graphs[i];
        J.p = p[i];
        J.q = q[i];
        J.anchor = resolve_anchor(graphs[i], p[i], q[i], 0);
        jobs.push_back(J);
        slot.push_back(i);
    }
    t_launches = 0;
    Timer tm;
    tm.init(false);
    if (!jobs.empty()) {
        gbc_status s = run_jobs(ctx, ctx->lane, ctx->budget, jobs, nullptr, false, tm, nullptr);
        if (s != GBC_OK) return s;
    }
    for (size_t j = 0; j < jobs.size(); ++j) {
        per_job[slot[j]] = jobs[j].st;
        if (jobs[j].st == GBC_OK) out[slot[j]] = gbc_u128{jobs[j].h.acc[0], jobs[j].h.acc[1]};
        else fail(jobs[j].st, "%s", jobs[j].err);
    }
    return GBC_OK;
}

extern "C" gbc_status gbc_count(gbc_graph_t g, int p, int q, gbc_u128 *out) {
    return count_impl(g, p, q, nullptr, out, nullptr, 0, nullptr);
}

extern "C" gbc_status gbc_count_ex(gbc_graph_t g, int p, int q, const gbc_count_options *opt, gbc_u128 *out,
                                   gbc_count_info *info) {
    gbc_u128 tmp;
    return count_impl(g, p, q, opt, out ? out : &tmp, info, 0, nullptr);
}

extern "C" gbc_status gbc_count_per_root(gbc_graph_t g, int p, int q, int anchor, gbc_u128 *per_root,
                                         gbc_u128 *total) {
    if (!g || !per_root || !total) return fail(GBC_ERR_ARG, "gbc_count_per_root: null argument");
    if (anchor != GBC_ANCHOR_U && anchor != GBC_ANCHOR_V) return fail(GBC_ERR_ARG, "gbc_count_per_root: anchor must be U or V");
    const int64_t nA = anchor == GBC_ANCHOR_U ? g->nU : g->nV;
    cudaStream_t st = g->ctx->lane.st;
    CK(cudaSetDevice(g->ctx->device));
    unsigned long long *d = nullptr;
    CK(cudaMallocAsync((void **)&d, (size_t)std::max<int64_t>(nA, 1) * 16, st));
    CK(cudaMemsetAsync(d, 0, (size_t)std::max<int64_t>(nA, 1) * 16, st));
    gbc_status s = count_impl(g, p, q, nullptr, total, nullptr, anchor, d);
    if (s == GBC_OK && nA > 0) {
        // per library id on the device; the caller's ids on the host
        std::vector<gbc_u128> tmp((size_t)nA);
        cudaError_t e = cudaMemcpyAsync(tmp.data(), d, (size_t)nA * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            s = fail(GBC_ERR_CUDA, "gbc_count_per_root: %s", cudaGetErrorString(e));
        } else {
            const std::vector<int32_t> &caller = anchor == GBC_ANCHOR_U ? g->callerU_h : g->callerV_h;
            for (int64_t i = 0; i < nA; ++i) per_root[caller[i]] = tmp[i];
        }
    }
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
    return s;
}

// ---------------------------------------------------------------------------
// Listing mode (Alg. 1 outputs the bicliques themselves).  gbc_list_begin sizes
// every root's records with one pass of the listing kernel; each
// gbc_list_next writes the records of the next roots whose records fit in the
// caller's buffer, so the caller drains the listing at its own pace.
struct gbc_lister_s {
    gbc_graph_s *g = nullptr;
    int p = 0, q = 0, anchor = 0;
    int64_t nA = 0;
    std::vector<int64_t> sizes;  // (words, records) per root, library ids
    int64_t next = 0;            // first root not yet written
};

static gbc_status run_list_job(gbc_lister_s *l, int mode, int32_t begin, int32_t end,
                               const std::vector<int64_t> *offsets, int32_t *out) {
    gbc_graph_s *g = l->g;
    gbc_ctx_s *ctx = g->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    std::vector<Job> jobs(1);
    Job &J = jobs[0];
    J.g = g;
    J.p = l->p;
    J.q = l->q;
    J.anchor = l->anchor;
    J.list_mode = mode;
    J.list_begin = begin;
    J.list_end = end;
    J.list_sizes = &l->sizes;
    J.list_offsets = offsets;
    J.list_out = out;
    Timer tm;
    tm.init(false);
    const gbc_status s = run_jobs(ctx, ctx->lane, ctx->budget, jobs, nullptr, false, tm, nullptr);
    if (s != GBC_OK) return s;
    if (J.st != GBC_OK) return fail(J.st, "%s", J.err);
    return GBC_OK;
}

extern "C" gbc_status gbc_list_begin(gbc_graph_t g, int p, int q, int anchor, gbc_lister_t *out,
                                     int64_t *total_words, int64_t *total_records, int64_t *max_root_words) {
    if (!g || !out) return fail(GBC_ERR_ARG, "gbc_list_begin: null argument");
    if (p < 1 || q < 1 || p > GBC_MAX_PQ || q > GBC_MAX_PQ)
        return fail(GBC_ERR_ARG, "gbc_list_begin: p=%d q=%d outside [1, %d]", p, q, GBC_MAX_PQ);
    if (anchor == GBC_ANCHOR_AUTO) anchor = GBC_ANCHOR_U;
    if (anchor != GBC_ANCHOR_U && anchor != GBC_ANCHOR_V) return fail(GBC_ERR_ARG, "gbc_list_begin: bad anchor %d", anchor);
    gbc_lister_s *l = new gbc_lister_s();
    l->g = g;
    l->p = p;
    l->q = q;
    l->anchor = anchor;
    l->nA = anchor == GBC_ANCHOR_U ? g->nU : g->nV;
    const gbc_status s = run_list_job(l, 1, 0, (int32_t)l->nA, nullptr, nullptr);
    if (s != GBC_OK) {
        delete l;
        return s;
    }
    int64_t w = 0, r = 0, mx = 0;
    for (int64_t u = 0; u < l->nA; ++u) {
        w += l->sizes[2 * u];
        r += l->sizes[2 * u + 1];
        mx = std::max(mx, l->sizes[2 * u]);
    }
    if (total_words) *total_words = w;
    if (total_records) *total_records = r;
    if (max_root_words) *max_root_words = mx;
    *out = l;
    return GBC_OK;
}

extern "C" gbc_status gbc_list_next(gbc_lister_t l, int32_t *buf_d, int64_t capacity_words, int64_t *words,
                                    int64_t *records, int *done) {
    if (!l || !words || !records || !done || capacity_words < 0 || (capacity_words > 0 && !buf_d))
        return fail(GBC_ERR_ARG, "gbc_list_next: bad argument");
    *words = 0;
    *records = 0;
    while (l->next < l->nA && l->sizes[2 * l->next] == 0) ++l->next;  // roots with nothing to list
    if (l->next >= l->nA) {
        *done = 1;
        return GBC_OK;
    }
    const int64_t begin = l->next;
    int64_t end = begin, w = 0, r = 0;
    while (end < l->nA && w + l->sizes[2 * end] <= capacity_words) {
        w += l->sizes[2 * end];
        r += l->sizes[2 * end + 1];
        ++end;
    }
    if (end == begin)
        return fail(GBC_ERR_OOM, "gbc_list_next: the next root's records need %lld words, more than the buffer's %lld",
                    (long long)l->sizes[2 * begin], (long long)capacity_words);
    std::vector<int64_t> offs((size_t)(end - begin));
    int64_t at = 0;
    for (int64_t u = begin; u < end; ++u) {
        offs[(size_t)(u - begin)] = at;
        at += l->sizes[2 * u];
    }
    const gbc_status s = run_list_job(l, 2, (int32_t)begin, (int32_t)end, &offs, buf_d);
    if (s != GBC_OK) return s;
    l->next = end;
    while (l->next < l->nA && l->sizes[2 * l->next] == 0) ++l->next;
    *words = w;
    *records = r;
    *done = l->next >= l->nA ? 1 : 0;
    return GBC_OK;
}

extern "C" void gbc_list_end(gbc_lister_t l) { delete l; }

// The autotuner: for each job it times the count from both anchors (the second
// bounded by the first's time) and keeps the faster one for later counts of the
// same (graph, p, q) on this context, plain or batched.  Anchors are the
// knob with the largest effect (5-10x for p = q >= 5 on power-law graphs);
// the cost model of pick_anchor is the starting point.
extern "C" gbc_status gbc_autotune(gbc_ctx_t ctx, int n, const gbc_graph_t *graphs, const int *p, const int *q,
                                   int time_limit_ms) {
    if (!ctx || n < 0 || (n > 0 && (!graphs || !p || !q))) return fail(GBC_ERR_ARG, "gbc_autotune: null argument");
    for (int i = 0; i < n; ++i) {
        if (!graphs[i] || graphs[i]->ctx != ctx || p[i] < 2 || q[i] < 2 || p[i] > GBC_MAX_PQ || q[i] > GBC_MAX_PQ)
            continue;  // one-sided sets have no choice to tune
        const TuneKey key{graphs[i], p[i], q[i]};
        {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            if (ctx->tuned_anchor.count(key)) continue;
        }
        const int first = pick_anchor(graphs[i], p[i], q[i]);
        const int second = first == GBC_ANCHOR_U ? GBC_ANCHOR_V : GBC_ANCHOR_U;
        gbc_count_options o;
        memset(&o, 0, sizeof o);
        o.anchor = first;
        o.time_limit_ms = time_limit_ms;
        gbc_count_info info;
        gbc_u128 v1, v2;
        gbc_status s1 = count_impl(graphs[i], p[i], q[i], &o, &v1, &info, 0, nullptr);
        if (s1 != GBC_OK && s1 != GBC_ERR_TIMEOUT) return s1;
        const float t1 = s1 == GBC_OK ? info.ms_total : 1e30f;
        o.anchor = second;
        o.time_limit_ms = s1 == GBC_OK ? std::max(1, (int)(t1 * 1.2f) + 1) : time_limit_ms;
        gbc_status s2 = count_impl(graphs[i], p[i], q[i], &o, &v2, &info, 0, nullptr);
        if (s2 != GBC_OK && s2 != GBC_ERR_TIMEOUT) return s2;
        const float t2 = s2 == GBC_OK ? info.ms_total : 1e30f;
        if (s1 == GBC_OK && s2 == GBC_OK && (v1.lo != v2.lo || v1.hi != v2.hi))
            return fail(GBC_ERR_CUDA, "gbc_autotune: the two anchors disagree on (%d,%d)", p[i], q[i]);
        const int best = t2 < t1 ? second : first;
        const float t_best = std::min(t1, t2);
        {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            ctx->tuned_anchor[key] = best;
        }
        // warps of the persistent enumeration launch: the default fills every SM
        // to its occupancy; fewer warps are kept only if they are >= 3% faster
        const int k = best == GBC_ANCHOR_U ? p[i] : q[i];
        if (k >= 4 && t_best < 1e29f) {
            o.anchor = best;
            float t_w = t_best;
            int w_best = 0;
            for (int frac : {2, 4}) {
                o.enum_warps = ctx->n_sms * 32 / frac;
                o.time_limit_ms = std::max(1, (int)(t_best * 1.2f) + 1);
                gbc_u128 v3;
                const gbc_status s3 = count_impl(graphs[i], p[i], q[i], &o, &v3, &info, 0, nullptr);
                if (s3 == GBC_ERR_TIMEOUT) continue;
                if (s3 != GBC_OK) return s3;
                const gbc_u128 &vb = best == first ? v1 : v2;
                if (v3.lo != vb.lo || v3.hi != vb.hi)
                    return fail(GBC_ERR_CUDA, "gbc_autotune: warp counts disagree on (%d,%d)", p[i], q[i]);
                if (info.ms_total < 0.97f * t_w) {
                    t_w = info.ms_total;
                    w_best = o.enum_warps;
                }
            }
            o.enum_warps = 0;
            if (w_best > 0) {
                std::lock_guard<std::mutex> lk(ctx->tune_mu);
                ctx->tuned_warps[key] = w_best;
            }
        }
    }
    return GBC_OK;
}

extern "C" int gbc_tuned_warps(gbc_graph_t g, int p, int q) {
    if (!g) return 0;
    std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
    auto it = g->ctx->tuned_warps.find(TuneKey{g, p, q});
    return it == g->ctx->tuned_warps.end() ? 0 : it->second;
}

extern "C" int gbc_tuned_anchor(gbc_graph_t g, int p, int q) {
    if (!g) return 0;
    std::lock_guard<std::mutex> lk(g->ctx->tune_mu);
    auto it = g->ctx->tuned_anchor.find(TuneKey{g, p, q});
    return it == g->ctx->tuned_anchor.end() ? 0 : it->second;
}

// ---------------------------------------------------------------------------
// Serving: gbc_submit / gbc_poll (continuous batching).
//
// Requests wait in a FIFO queue.  Each worker thread has its own lane of
// streams; a free worker takes waiting requests as one batch while their
// scratch footprints (footprint_of: exact once the same count has run, else an
// upper bound from the graph's wedge sums) fit in the part of the context's
// budget that no other batch holds.  A request that fits nowhere waits until
// running batches give memory back; one that exceeds the whole budget runs
// alone.  The head of the queue is passed over by smaller requests at most
// kMaxSkips times, so it is never starved.  Every request is released as soon
// as its own count is done -- counts that finish early in the pipeline at the
// host synchronisations, the others through the device's completion records --
// not when the whole batch ends, and its memory returns when the batch ends.
// Submission refuses a request when max_queue requests are already waiting.
constexpr int kMaxSkips = 16;

struct Request {
    uint64_t ticket = 0;
    gbc_graph_s *g = nullptr;
    int p = 0, q = 0, time_limit_ms = 0;
    size_t foot = 0;        // scratch bytes reserved for it (footprint_of)
    int skipped = 0;        // times a later request was admitted ahead of it
    bool done = false;
    gbc_status st = GBC_OK;
    gbc_u128 val{0, 0};
    char err[256] = "";
};

struct Server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    int max_batch = 256, max_queue = 4096, time_limit_ms = 0;
    size_t budget = 0;          // scratch budget shared by the workers' batches
    size_t in_flight = 0;       // scratch reserved by the batches on the device
    gbc_serve_stats stats{};
    int running = 0;            // batches on the device
    std::vector<std::thread> threads;
    std::vector<Lane> lanes;
    std::vector<cudaStream_t> own_streams;
};

// Takes the next batch for a worker (caller holds sv->mu); empty if nothing fits.
static std::vector<Request *> take_batch(Server *sv, size_t &reserved) {
    std::vector<Request *> batch;
    reserved = 0;
    for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)batch.size() < sv->max_batch;) {
        Request *r = *it;
        const bool alone = sv->in_flight == 0 && batch.empty();
        const bool fits = sv->in_flight + reserved + r->foot <= sv->budget;
        if (alone || fits) {
            batch.push_back(r);
            reserved += std::min(r->foot, sv->budget);  // alone, it may use the whole budget and no more
            it = sv->pending.erase(it);
            continue;
        }
        if (it == sv->pending.begin()) {
            // the head does not fit: later requests may pass it a bounded number of times
            if (++r->skipped > kMaxSkips) break;
        }
        ++it;
    }
    return batch;
}

static void serve_loop(gbc_ctx_s *ctx, Server *sv, int w) {
    cudaSetDevice(ctx->device);
    while (true) {
        std::vector<Request *> batch;
        size_t reserved = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            while (true) {
                if (sv->pending.empty()) {
                    if (sv->stop) return;  // stopping and drained
                } else {
                    batch = take_batch(sv, reserved);
                    if (!batch.empty()) break;
                }
                sv->cv_work.wait(lk);
            }
            sv->in_flight += reserved;
            sv->running += 1;
            sv->stats.batches += 1;
            sv->stats.admitted += (int64_t)batch.size();
            sv->stats.peak_in_flight_bytes = std::max<int64_t>(sv->stats.peak_in_flight_bytes, (int64_t)sv->in_flight);
            sv->stats.peak_running_batches = std::max<int32_t>(sv->stats.peak_running_batches, sv->running);
        }
        std::vector<Job> jobs(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) {
            jobs[i].g = batch[i]->g;
            jobs[i].p = batch[i]->p;
            jobs[i].q = batch[i]->q;
            jobs[i].time_limit_ms = batch[i]->time_limit_ms;
            jobs[i].anchor = resolve_anchor(batch[i]->g, batch[i]->p, batch[i]->q, 0);
        }
        // finished[i]: request i was handed over (a poll may have freed it since)
        std::vector<char> finished(batch.size(), 0);
        const DoneFn on_done = [&](int i, gbc_status st, gbc_u128 v, const char *msg) {
            std::lock_guard<std::mutex> lk(sv->mu);
            finished[i] = 1;
            Request *r = batch[i];
            r->st = st;
            r->val = v;
            snprintf(r->err, sizeof r->err, "%s", msg);
            r->done = true;
            sv->cv_done.notify_all();
        };
        Timer tm;
        tm.init(false);
        // a batch may use what it reserved (a request too large for any share runs alone on the whole budget)
        const size_t run_budget = reserved;
        const gbc_status s = run_jobs(ctx, sv->lanes[w], run_budget, jobs, nullptr, false, tm, nullptr, &on_done);
        const char *batch_err = s == GBC_OK ? "" : gbc_last_error();
        std::lock_guard<std::mutex> lk(sv->mu);
        for (size_t i = 0; i < batch.size(); ++i) {
            if (finished[i]) continue;
            Request *r = batch[i];
            r->st = s != GBC_OK ? s : GBC_ERR_CUDA;
            snprintf(r->err, sizeof r->err, "%s", s != GBC_OK ? batch_err : "gbc_serve: request not completed");
            r->done = true;
        }
        sv->in_flight -= reserved;
        sv->running -= 1;
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();  // memory came back: waiting requests may fit now
    }
}

static void stop_server(gbc_ctx_s *ctx) {
    Server *sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->threads) t.join();
    for (auto &l : sv->lanes) l.destroy();
    for (auto s : sv->own_streams) cudaStreamDestroy(s);
    for (auto &kv : sv->all) delete kv.second;
    delete sv;
    ctx->server = nullptr;
}

extern "C" gbc_status gbc_serve_start(gbc_ctx_t ctx, int workers, int max_batch, int max_queue, int time_limit_ms) {
    if (!ctx || workers < 0 || max_batch < 0 || max_queue < 0 || time_limit_ms < 0)
        return fail(GBC_ERR_ARG, "gbc_serve_start: bad argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->server) return fail(GBC_ERR_ARG, "gbc_serve_start: already serving");
    CK(cudaSetDevice(ctx->device));
    // the context's budget, but no more than the device memory free now (the
    // resident graphs were loaded after the budget was set)
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    Server *sv = new Server();
    const int nw = workers ? workers : 4;
    sv->max_batch = max_batch ? max_batch : 256;
    sv->max_queue = max_queue ? max_queue : 4096;
    sv->time_limit_ms = time_limit_ms;
    sv->budget = std::min(ctx->budget, (size_t)(0.9 * (double)free_b));
    sv->lanes.resize(nw);
    for (int w = 0; w < nw; ++w) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = sv->lanes[w].create(s);
        if (e != cudaSuccess) {
            for (auto &l : sv->lanes) l.destroy();
            for (auto x : sv->own_streams) cudaStreamDestroy(x);
            delete sv;
            return fail(GBC_ERR_CUDA, "gbc_serve_start: %s", cudaGetErrorString(e));
        }
        sv->own_streams.push_back(s);
    }
    ctx->server = sv;
    for (int w = 0; w < nw; ++w) sv->threads.emplace_back(serve_loop, ctx, sv, w);
    return GBC_OK;
}

extern "C" gbc_status gbc_serve_stop(gbc_ctx_t ctx) {
    if (!ctx) return fail(GBC_ERR_ARG, "gbc_serve_stop: null context");
    stop_server(ctx);
    return GBC_OK;
}

extern "C" gbc_status gbc_serve_stats_get(gbc_ctx_t ctx, gbc_serve_stats *out) {
    if (!ctx || !out) return fail(GBC_ERR_ARG, "gbc_serve_stats_get: null argument");
    Server *sv = ctx->server;
    if (!sv) return fail(GBC_ERR_ARG, "gbc_serve_stats_get: not serving");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->budget_bytes = (int64_t)sv->budget;
    return GBC_OK;
}

extern "C" gbc_status gbc_footprint(gbc_graph_t g, int p, int q, size_t *bytes, int *exact) {
    if (!g || !bytes) return fail(GBC_ERR_ARG, "gbc_footprint: null argument");
    if (p < 1 || q < 1 || p > GBC_MAX_PQ || q > GBC_MAX_PQ)
        return fail(GBC_ERR_ARG, "gbc_footprint: p=%d q=%d outside [1, %d]", p, q, GBC_MAX_PQ);
    *bytes = footprint_of(g, resolve_anchor(g, p, q, 0), p, q, exact);
    return GBC_OK;
}

extern "C" gbc_status gbc_submit(gbc_ctx_t ctx, gbc_graph_t g, int p, int q, uint64_t *ticket) {
    if (!ctx || !g || !ticket || g->ctx != ctx) return fail(GBC_ERR_ARG, "gbc_submit: bad argument");
    if (p < 1 || q < 1 || p > GBC_MAX_PQ || q > GBC_MAX_PQ)
        return fail(GBC_ERR_ARG, "gbc_submit: p=%d q=%d outside [1, %d]", p, q, GBC_MAX_PQ);
    if (!ctx->server) {
        gbc_status s = gbc_serve_start(ctx, 0, 0, 0, 0);
        if (s != GBC_OK && !ctx->server) return s;
    }
    Server *sv = ctx->server;
    const size_t foot = footprint_of(g, resolve_anchor(g, p, q, 0), p, q, nullptr);
    std::lock_guard<std::mutex> lk(sv->mu);
    if ((int)sv->pending.size() >= sv->max_queue) {
        sv->stats.rejected += 1;
        return fail(GBC_ERR_REJECTED, "gbc_submit: %d requests already waiting", (int)sv->pending.size());
    }
    Request *r = new Request();
    r->ticket = sv->next_ticket++;
    r->g = g;
    r->p = p;
    r->q = q;
    r->time_limit_ms = sv->time_limit_ms;
    r->foot = foot;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    sv->stats.submitted += 1;
    *ticket = r->ticket;
    sv->cv_work.notify_one();
    return GBC_OK;
}

extern "C" gbc_status gbc_poll(gbc_ctx_t ctx, uint64_t ticket, int timeout_ms, gbc_u128 *out) {
    if (!ctx || !out) return fail(GBC_ERR_ARG, "gbc_poll: null argument");
    Server *sv = ctx->server;
    if (!sv) return fail(GBC_ERR_ARG, "gbc_poll: not serving");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(GBC_ERR_ARG, "gbc_poll: unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (!r->done) {
        if (timeout_ms > 0)
            sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
        else if (timeout_ms < 0)
            sv->cv_done.wait(lk, [&] { return r->done; });
        if (!r->done) return GBC_PENDING;
    }
    const gbc_status s = r->st;
    if (s == GBC_OK) *out = r->val;
    else fail(s, "%s", r->err);
    sv->all.erase(it);
    delete r;
    return s;
}
