// Batched ALI over many independent models (uneven sizes) with one persistent formal-solve
// launch per iteration and the iteration captured as a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include "common.cuh"

namespace {

// Total expanded points over all rays of each origin point (the cost of its work items).
__global__ void k_origin_cost(int64_t n, int R, const int64_t *ray_off, const int32_t *xcum, int64_t *cost) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    int64_t s = 0;
    for (int r = 0; r < R; r++) {
        const int64_t a = ray_off[o * R + r], b = ray_off[o * R + r + 1];
        s += (b > a ? xcum[b - 1] : 0) + 1;
    }
    cost[o] = s;
}

__global__ void k_copy_if_active(const int32_t *active, int64_t m, const double *src, double *dst) {
    if (!*active) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Gathers each model's (max change bits, fallback count, non-finite count).
__global__ void k_gather_scal(int nm, unsigned long long *const *scal, unsigned long long *out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nm) return;
    out[3 * m] = scal[m][0];
    out[3 * m + 1] = scal[m][1];
    out[3 * m + 2] = scal[m][2];
}

struct Item {
    int32_t model;
    int32_t local;
};

}  // namespace

struct mg_batch {
    int n_models = 0;
    std::vector<mg_ctx *> models;
    int device = 0;
    cudaStream_t stream = nullptr;
    int L = 0, Q = 0;
    int variant = -1, grid = 0, sorted = 1;
    // work-item lists per lines-per-warp value G (index G, 1 <= G <= kMaxG), natural and
    // cost order
    static constexpr int kMaxG = 4;
    int64_t n_items_g[kMaxG + 1] = {};
    void *d_args = nullptr;
    Item *d_items_g[kMaxG + 1][2] = {};
    unsigned long long *d_counter = nullptr;
    int32_t *d_active = nullptr;
    int32_t *h_active = nullptr;         // pinned
    unsigned long long **d_scal_ptrs = nullptr;
    unsigned long long *d_scal_all = nullptr, *h_scal_all = nullptr;   // pinned host copy
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_order = nullptr;      // orders the batch stream after each model's stream
    std::string err;
    int num_sms = 152;
};

static int bfail(mg_batch *b, int code, const std::string &m) {
    if (b) b->err = m;
    return code;
}

#define B_CUDA(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return bfail(b, MG_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// Work items (model, origin * L + first line of the group) for every lines-per-warp value
// G of the launch variants (1, 2 and 4), each in cost order (longest first) and in natural
// order.
static int build_items(mg_batch *b) {
    std::vector<int64_t> cost_all;
    std::vector<std::pair<int32_t, int64_t>> who;   // (model, origin)
    for (int m = 0; m < b->n_models; m++) {
        mg_ctx *c = b->models[m];
        int64_t *d_cost = nullptr;
        B_CUDA(cudaMalloc(&d_cost, sizeof(int64_t) * c->n));
        k_origin_cost<<<(unsigned)((c->n + 255) / 256), 256, 0, b->stream>>>(c->n, c->R, c->d_ray_off, c->d_xcum, d_cost);
        std::vector<int64_t> cost(c->n);
        B_CUDA(cudaMemcpyAsync(cost.data(), d_cost, sizeof(int64_t) * c->n, cudaMemcpyDeviceToHost, b->stream));
        B_CUDA(cudaStreamSynchronize(b->stream));
        cudaFree(d_cost);
        for (int64_t o = 0; o < c->n; o++) {
            cost_all.push_back(cost[o]);
            who.push_back({m, o});
        }
    }
    std::vector<size_t> order(who.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost_all[x] > cost_all[y]; });
    for (int G = 1; G <= mg_batch::kMaxG; G *= 2) {
        std::vector<Item> nat, srt;
        for (size_t i = 0; i < who.size(); i++)
            for (int l0 = 0; l0 < b->L; l0 += G) nat.push_back(Item{who[i].first, (int32_t)(who[i].second * b->L + l0)});
        for (size_t i : order)
            for (int l0 = 0; l0 < b->L; l0 += G) srt.push_back(Item{who[i].first, (int32_t)(who[i].second * b->L + l0)});
        b->n_items_g[G] = (int64_t)nat.size();
        for (int k = 0; k < 2; k++) {
            Item *&d = b->d_items_g[G][k];
            if (d) cudaFree(d);
            B_CUDA(cudaMalloc(&d, sizeof(Item) * nat.size()));
            B_CUDA(cudaMemcpyAsync(d, k ? srt.data() : nat.data(), sizeof(Item) * nat.size(), cudaMemcpyHostToDevice,
                                   b->stream));
        }
        B_CUDA(cudaStreamSynchronize(b->stream));
    }
    return MG_OK;
}

static int launch_solve(mg_batch *b) {
    B_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->stream));
    int v = b->variant >= 0 ? b->variant : mg_variant_default(b->L, b->Q);
    for (auto *c : b->models) v = mg_variant_effective(c, v);   // no skipping under a large opacity floor
    const int grid = b->grid > 0 ? b->grid : b->num_sms * mg_variant_minb(v);
    const int G = mg_variant_g(v);
    if (G < 1 || G > mg_batch::kMaxG || !b->d_items_g[G][0] || !b->d_items_g[G][1])
        return bfail(b, MG_ERR_ARG, "batch: no work-item list for this launch variant");
    int rc = mg_batch_launch(v, grid, b->d_args, b->d_items_g[G][b->sorted ? 1 : 0], b->n_items_g[G],
                             b->d_counter, b->d_active, b->stream);
    if (rc) return bfail(b, rc, "batch: persistent formal-solve launch failed");
    return MG_OK;
}

// Points every model's context at the batch stream (and back). The batch stream first
// waits for the work already queued on each model's own stream (population uploads,
// initialisations), which it would otherwise overtake.
struct StreamSwap {
    mg_batch *b;
    std::vector<cudaStream_t> saved;
    std::vector<int32_t> prof;
    explicit StreamSwap(mg_batch *bb) : b(bb) {
        for (auto *c : b->models) {
            if (c->stream != b->stream && cudaEventRecord(b->ev_order, c->stream) == cudaSuccess)
                cudaStreamWaitEvent(b->stream, b->ev_order, 0);
            saved.push_back(c->stream);
            prof.push_back(c->opt.profile);
            c->stream = b->stream;
            c->opt.profile = 0;
        }
    }
    ~StreamSwap() {
        for (size_t i = 0; i < b->models.size(); i++) {
            b->models[i]->stream = saved[i];
            b->models[i]->opt.profile = prof[i];
        }
    }
};

extern "C" int mg_batch_create(mg_batch **out, int32_t n_models, mg_ctx *const *models) {
    if (!out || n_models < 1 || !models) return MG_ERR_ARG;
    *out = nullptr;
    mg_batch *b = new mg_batch();
    b->n_models = n_models;
    b->models.assign(models, models + n_models);
    mg_ctx *c0 = models[0];
    if (!c0) { delete b; return MG_ERR_ARG; }
    b->device = c0->device;
    b->L = c0->n_lines;
    b->Q = c0->Q;
    for (auto *c : b->models) {
        if (!c || c->device != b->device || c->opt.precision != MG_MIXED || c->n_lines != b->L || c->Q != b->Q) {
            c0->err = "mg_batch_create: models must share the device, MG_MIXED precision, n_lines and n_q";
            delete b;
            return MG_ERR_ARG;
        }
        int rc = mg_ensure_solve_state(c);
        if (rc) { delete b; return rc; }
    }
    cudaSetDevice(b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return MG_ERR_CUDA; }
    if (cudaEventCreateWithFlags(&b->ev_order, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(b->stream);
        delete b;
        return MG_ERR_CUDA;
    }
    const size_t asz = mg_mixargs_size();
    std::vector<unsigned char> args(asz * n_models);
    for (int m = 0; m < n_models; m++) {
        int rc = mg_fill_mixargs(b->models[m], args.data() + asz * m);
        if (rc) { mg_batch_destroy(b); return rc; }
    }
    std::vector<unsigned long long *> sp(n_models);
    for (int m = 0; m < n_models; m++) sp[m] = b->models[m]->d_scal;
    if (cudaMalloc(&b->d_args, asz * n_models) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&b->d_active, sizeof(int32_t) * n_models) != cudaSuccess ||
        cudaMallocHost(&b->h_active, sizeof(int32_t) * n_models) != cudaSuccess ||
        cudaMalloc(&b->d_scal_ptrs, sizeof(void *) * n_models) != cudaSuccess ||
        cudaMalloc(&b->d_scal_all, 3 * sizeof(unsigned long long) * n_models) != cudaSuccess ||
        cudaMallocHost(&b->h_scal_all, 3 * sizeof(unsigned long long) * n_models) != cudaSuccess) {
        mg_batch_destroy(b);
        return MG_ERR_OOM;
    }
    for (int m = 0; m < n_models; m++) b->h_active[m] = 1;
    cudaMemcpyAsync(b->d_args, args.data(), asz * n_models, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_scal_ptrs, sp.data(), sizeof(void *) * n_models, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int32_t) * n_models, cudaMemcpyHostToDevice, b->stream);
    for (auto *c : b->models)   // the ray stores may still be in flight on the models' streams
        if (cudaEventRecord(b->ev_order, c->stream) == cudaSuccess) cudaStreamWaitEvent(b->stream, b->ev_order, 0);
    int rc = build_items(b);
    if (rc) { mg_batch_destroy(b); return rc; }
    *out = b;
    return MG_OK;
}

extern "C" int mg_batch_destroy(mg_batch *b) {
    if (!b) return MG_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int G = 1; G <= mg_batch::kMaxG; G++)
        for (int k = 0; k < 2; k++) cudaFree(b->d_items_g[G][k]);
    cudaFree(b->d_args); cudaFree(b->d_counter);
    cudaFree(b->d_active); cudaFree(b->d_scal_ptrs); cudaFree(b->d_scal_all);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_scal_all) cudaFreeHost(b->h_scal_all);
    if (b->ev_order) cudaEventDestroy(b->ev_order);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return MG_OK;
}

extern "C" const char *mg_batch_last_error(const mg_batch *b) { return b ? b->err.c_str() : "null batch"; }

// Line data of every model, then one persistent formal-solve launch for all of them.
static int enqueue_formal_solve(mg_batch *b) {
    for (auto *c : b->models) {
        cudaMemsetAsync(c->d_scal + 4, 0, sizeof(unsigned long long), b->stream);
        int rc = mg_launch_line_data(c);
        if (rc) return bfail(b, rc, "batch: line data launch failed");
    }
    return launch_solve(b);
}

extern "C" int mg_batch_formal_solve(mg_batch *b) {
    if (!b) return MG_ERR_ARG;
    cudaSetDevice(b->device);
    StreamSwap sw(b);
    int rc = enqueue_formal_solve(b);
    if (rc) return rc;
    B_CUDA(cudaStreamSynchronize(b->stream));
    for (auto *c : b->models) c->have_rad = true;
    return MG_OK;
}

// One ALI iteration for all active models: line data, persistent formal solve,
// statistical equilibrium into pops_new, copy back, gather of the convergence words.
static int enqueue_iteration(mg_batch *b) {
    int rc = enqueue_formal_solve(b);
    if (rc) return rc;
    for (int m = 0; m < b->n_models; m++) {
        mg_ctx *c = b->models[m];
        cudaMemsetAsync(c->d_scal, 0, 3 * sizeof(unsigned long long), b->stream);
        if ((rc = mg_launch_stateq_into(c, c->d_pops, c->d_pops_new, b->d_active + m))) return bfail(b, rc, "batch: stateq");
        const int64_t mm = c->n * c->n_lev;
        k_copy_if_active<<<(unsigned)std::min<int64_t>(1024, (mm + 255) / 256), 256, 0, b->stream>>>(
            b->d_active + m, mm, c->d_pops_new, c->d_pops);
    }
    k_gather_scal<<<(b->n_models + 127) / 128, 128, 0, b->stream>>>(b->n_models, b->d_scal_ptrs, b->d_scal_all);
    cudaMemcpyAsync(b->h_scal_all, b->d_scal_all, 3 * sizeof(unsigned long long) * b->n_models,
                    cudaMemcpyDeviceToHost, b->stream);
    B_CUDA(cudaGetLastError());
    return MG_OK;
}

extern "C" int mg_batch_iterate(mg_batch *b, mg_ali_report *reps) {
    if (!b) return MG_ERR_ARG;
    cudaSetDevice(b->device);
    StreamSwap sw(b);
    auto t0 = std::chrono::steady_clock::now();
    std::vector<mg_ali_report> r(b->n_models);
    for (int m = 0; m < b->n_models; m++) {
        std::memset(&r[m], 0, sizeof(mg_ali_report));
        b->h_active[m] = 1;
    }
    B_CUDA(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int32_t) * b->n_models, cudaMemcpyHostToDevice, b->stream));
    if (!b->exec) {
        cudaGraph_t g;
        B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_iteration(b);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return bfail(b, MG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    const int max_iter = b->models[0]->opt.max_iter;
    int n_active = b->n_models;
    std::vector<int> nh(b->n_models, 0);   // iterates in each model's Ng history
    for (int it = 0; it < max_iter && n_active > 0; it++) {
        B_CUDA(cudaGraphLaunch(b->exec, b->stream));
        B_CUDA(cudaStreamSynchronize(b->stream));
        bool changed = false;
        for (int m = 0; m < b->n_models; m++) {
            if (!b->h_active[m]) continue;
            mg_ctx *c = b->models[m];
            double ch;
            std::memcpy(&ch, &b->h_scal_all[3 * m], 8);
            r[m].iterations++;
            r[m].last_change = ch;
            r[m].n_fallback += (int64_t)b->h_scal_all[3 * m + 1];
            if (b->h_scal_all[3 * m + 2]) return bfail(b, MG_ERR_NUMERIC, "batch: non-finite populations");
            if (ch < c->opt.tol) {
                r[m].converged = 1;
                b->h_active[m] = 0;
                n_active--;
                changed = true;
                continue;
            }
            // Ng acceleration of this model, as in mg_iterate (outside the graph: the
            // history ring rotates and the step's acceptance is read on the host)
            if (c->opt.ng_period > 0) {
                int rc = mg_launch_push_history(c);
                if (rc) return bfail(b, rc, "batch: Ng history");
                if (nh[m] < 4) nh[m]++;
                if (nh[m] == 4 && (it + 1) % c->opt.ng_period == 0) {
                    int acc = 0;
                    if ((rc = mg_launch_ng(c, &acc))) return bfail(b, rc, "batch: Ng step");
                    r[m].ng_steps += acc;
                    nh[m] = 0;
                }
            }
        }
        if (changed)
            B_CUDA(cudaMemcpyAsync(b->d_active, b->h_active, sizeof(int32_t) * b->n_models, cudaMemcpyHostToDevice, b->stream));
    }
    B_CUDA(cudaStreamSynchronize(b->stream));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int m = 0; m < b->n_models; m++) {
        r[m].seconds = sec;
        all = all && r[m].converged;
        b->models[m]->have_rad = false;
        b->models[m]->have_pops = true;
        if (reps) reps[m] = r[m];
    }
    return all ? MG_OK : bfail(b, MG_ERR_NOT_CONVERGED, "batch: some models did not converge");
}

// Times every valid launch variant of the persistent kernel, with the queue sorted by
// cost and unsorted, and keeps the fastest (one warm-up, best of reps).
extern "C" int mg_batch_set_variant(mg_batch *b, int32_t variant, int32_t sorted) {
    if (!b) return MG_ERR_ARG;
    if (variant != -1 && !mg_variant_valid(variant, b->L, b->Q))
        return bfail(b, MG_ERR_ARG, "mg_batch_set_variant: variant not valid for this batch's lines and bins");
    b->variant = variant;
    b->sorted = sorted ? 1 : 0;
    b->grid = 0;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    return MG_OK;
}

extern "C" int mg_batch_autotune(mg_batch *b, int32_t reps, int32_t *variant, int32_t *sorted, double *ms) {
    if (!b) return MG_ERR_ARG;
    cudaSetDevice(b->device);
    StreamSwap sw(b);
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    int rc0 = enqueue_formal_solve(b);   // line data for every model
    if (rc0) return rc0;
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = -1, bs = 1;
    for (int v = 0; v < mg_variant_count(); v++) {
        if (!mg_variant_valid(v, b->L, b->Q)) continue;
        for (int srt = 0; srt < 2; srt++) {
            b->variant = v;
            b->sorted = srt;
            b->grid = 0;
            float vb = 1e30f;
            for (int k = 0; k < reps + 1; k++) {
                cudaEventRecord(e0, b->stream);
                int rc = launch_solve(b);
                cudaEventRecord(e1, b->stream);
                if (rc) return rc;
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (k > 0) vb = std::min(vb, t);
            }
            if (vb < best) { best = vb; bv = v; bs = srt; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = bv;
    b->sorted = bs;
    for (auto *c : b->models) c->have_rad = true;
    if (variant) *variant = bv;
    if (sorted) *sorted = bs;
    if (ms) *ms = best;
    return MG_OK;
}

extern "C" int mg_batch_work_counts(const mg_batch *b, int64_t *solves, int64_t *updates) {
    if (!b) return MG_ERR_ARG;
    int64_t s = 0, u = 0;
    for (auto *c : b->models) {
        int64_t a = 0, d = 0;
        mg_work_counts(c, &a, &d);
        s += a;
        u += d;
    }
    if (solves) *solves = s;
    if (updates) *updates = u;
    return MG_OK;
}
