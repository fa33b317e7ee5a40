// K4 statistical equilibrium (eq. 'ourALI'), validity check (Sec. 6.1), convergence
// measure, LTE start and Ng acceleration (Sec. 3.4).
#include <cmath>
#include <cstring>
#include "common.cuh"
#include "stateq_common.cuh"

using namespace mg;

namespace {

// LTE (Boltzmann) populations n_i = n g_i exp(-E_i/kT) / sum_j g_j exp(-E_j/kT).
__global__ void k_lte(int64_t n, int nlev, const double *E, const double *g, const double *T, const double *nspec,
                      double *pops) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double ikT = 1.0 / (kKB * T[c]);
    double Z = 0.0;
    for (int i = 0; i < nlev; i++) Z += g[i] * exp(-E[i] * ikT);
    const double s = nspec[c] / Z;
    for (int i = 0; i < nlev; i++) pops[c * nlev + i] = s * g[i] * exp(-E[i] * ikT);
}

// Collision rates per point and level pair (i > j), stored as (down, up):
// C_ij = K_ij(T) n_coll with K interpolated linearly in T (constant beyond the grid), and
// C_ji = C_ij (g_i/g_j) exp(-(E_i - E_j)/kT) (detailed balance).
__global__ void k_collision_rates(int64_t n, int nlev, int nT, const double *E, const double *g,
                                  const double *Tg, const double *K, const double *T, const double *ncoll,
                                  double *coll) {
    const int npairs = nlev * (nlev - 1) / 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * npairs) return;
    const int64_t c = t / npairs;
    const int pr = (int)(t - c * npairs);
    int i = 1;
    while ((i + 1) * i / 2 <= pr) i++;
    const int j = pr - i * (i - 1) / 2;
    const double Tc = T[c];
    double Cd, Cu;
    collision_rates_pair(collision_k_down(K, pr, nT, Tg, Tc), ncoll[c], g[i], g[j], E[i], E[j], Tc, Cd, Cu);
    coll[2 * t] = Cd;
    coll[2 * t + 1] = Cu;
}

struct StateqArgs {
    int64_t n;
    int nlev, L;
    const LineConst *lc;
    const double *pops;      // old
    double *pops_new;
    const double *J, *Lc, *Jeff;
    const double *coll;      // [n][npairs][2]
    const double *nspec;
    unsigned long long *scal;   // [0] max change bits, [1] fallback count, [2] non-finite count
    const int32_t *active;      // optional: skip the whole launch when *active == 0
};

// Rates u->l = A (1 - L) + B_ul Jeff + C_ul, l->u = B_lu Jeff + C_lu (eq. 'ourALI');
// 1 - L is passed in directly (accumulated without cancellation by the formal solve).
template <int MAXLEV>
__device__ void build_rates(const StateqArgs &a, int64_t c, bool plain, double (&q)[MAXLEV][MAXLEV]) {
    const int n = a.nlev;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) q[i][j] = 0.0;
    line_rates<MAXLEV>(a.L, a.lc, a.J, a.Lc, a.Jeff, c, plain, q);
    const int npairs = n * (n - 1) / 2;
    const double *cr = a.coll + (size_t)c * npairs * 2;
    int pr = 0;
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++, pr++) {
            q[i][j] += cr[2 * pr];
            q[j][i] += cr[2 * pr + 1];
        }
}

template <int MAXLEV>
__global__ void k_stateq(StateqArgs a) {
    if (a.active && !*a.active) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double change = 0.0;
    unsigned long long fb = 0, bad = 0;
    if (c < a.n) {
        const int n = a.nlev;
        double q[MAXLEV][MAXLEV], pi[MAXLEV];
        build_rates<MAXLEV>(a, c, false, q);
        bool ok = gth_solve<MAXLEV>(n, q, pi) && valid_fractions<MAXLEV>(n, pi);
        if (!ok) {
            fb = 1;
            build_rates<MAXLEV>(a, c, true, q);
            ok = gth_solve<MAXLEV>(n, q, pi) && valid_fractions<MAXLEV>(n, pi);
            if (!ok) bad = 1;
        }
        const double ns = a.nspec[c];
        for (int i = 0; i < n; i++) {
            const double nw = ns * pi[i];
            const double od = a.pops[c * n + i];
            a.pops_new[c * n + i] = nw;
            if (nw >= 1e-10 * ns) {
                const double d = fabs(nw - od) / nw;
                if (d > change) change = d;
            }
        }
        if (!isfinite(change)) change = INFINITY;
    }
    // positive doubles order like their bit patterns: max over bits is deterministic
    unsigned long long bits = __double_as_longlong(change);
    for (int d = 16; d; d >>= 1) {
        unsigned long long o = __shfl_down_sync(0xffffffffu, bits, d);
        bits = o > bits ? o : bits;
        fb += __shfl_down_sync(0xffffffffu, fb, d);
        bad += __shfl_down_sync(0xffffffffu, bad, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&a.scal[0], bits);
        if (fb) atomicAdd(&a.scal[1], fb);
        if (bad) atomicAdd(&a.scal[2], bad);
    }
}

// ---------------------------------------------------------------- Ng acceleration
// History of fractional populations x = n_i / n_spec (uniform weights over levels).
__global__ void k_push_history(int64_t m, int nlev, const double *pops, const double *nspec, double *dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    dst[t] = pops[t] / nspec[t / nlev];
}

constexpr int kNgBlocks = 512;
constexpr int kNgThreads = 256;

// Partial sums of the Ng normal equations with D_i = x_i - x_{i+1}, Q_j = D_0 - D_j:
// a11 = <Q1,Q1>, a12 = <Q1,Q2>, a22 = <Q2,Q2>, b1 = <Q1,D0>, b2 = <Q2,D0>. Each block
// writes its partials; a fixed-order sum follows, so the result is reproducible.
__global__ void k_ng_dots(int64_t m, const double *x0, const double *x1, const double *x2, const double *x3,
                          double *part) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const double D0 = x0[t] - x1[t], D1 = x1[t] - x2[t], D2 = x2[t] - x3[t];
        const double Q1 = D0 - D1, Q2 = D0 - D2;
        s[0] += Q1 * Q1; s[1] += Q1 * Q2; s[2] += Q2 * Q2; s[3] += Q1 * D0; s[4] += Q2 * D0;
    }
    __shared__ double sh[5][kNgThreads];
    for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kNgThreads / 2; w; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 5; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; k++) part[5 * blockIdx.x + k] = sh[k][0];
}

// Sums the partials in block order, solves the 2x2 system and forms
// x = (1 - a1 - a2) x0 + a1 x1 + a2 x2 in tmp; flags a singular system or a negative value.
__global__ void k_ng_apply(int64_t m, int nlev, const double *part, int nparts, const double *x0, const double *x1,
                           const double *x2, const double *nspec, double *tmp, unsigned long long *flag) {
    __shared__ double coef[2];
    __shared__ int singular;
    if (threadIdx.x == 0) {
        double s[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < nparts; b++)
            for (int k = 0; k < 5; k++) s[k] += part[5 * b + k];
        const double det = s[0] * s[2] - s[1] * s[1];
        singular = !(det != 0.0 && isfinite(det));
        coef[0] = singular ? 0.0 : (s[3] * s[2] - s[4] * s[1]) / det;
        coef[1] = singular ? 0.0 : (s[0] * s[4] - s[1] * s[3]) / det;
        if (singular && blockIdx.x == 0) atomicOr(flag, 1ull);
    }
    __syncthreads();
    if (singular) return;
    const double a1 = coef[0], a2 = coef[1];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = (1.0 - a1 - a2) * x0[t] + a1 * x1[t] + a2 * x2[t];
        if (!(x >= 0.0)) atomicOr(flag, 2ull);
        tmp[t] = x * nspec[t / nlev];
    }
}

}  // namespace

int mg_launch_lte(mg_ctx *ctx) {
    MgTimed t(ctx, "lte");
    k_lte<<<(unsigned)((ctx->n + 127) / 128), 128, 0, ctx->stream>>>(ctx->n, ctx->n_lev, ctx->d_E, ctx->d_g,
                                                                      ctx->d_T, ctx->d_nspec, ctx->d_pops);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_collision_rates(mg_ctx *ctx) {
    const int npairs = ctx->n_lev * (ctx->n_lev - 1) / 2;
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_coll, (size_t)ctx->n * npairs * 2))) return rc;
    const int64_t m = ctx->n * npairs;
    k_collision_rates<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->n, ctx->n_lev, ctx->n_T, ctx->d_E, ctx->d_g, ctx->d_Tgrid, ctx->d_Kdown, ctx->d_T, ctx->d_ncoll,
        ctx->d_coll);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_stateq(mg_ctx *ctx) {
    StateqArgs a{};
    a.n = ctx->n; a.nlev = ctx->n_lev; a.L = ctx->n_lines; a.lc = ctx->d_lines;
    a.pops = ctx->d_pops; a.pops_new = ctx->d_pops_new; a.J = ctx->d_J; a.Lc = ctx->d_Lc; a.Jeff = ctx->d_Jeff;
    a.coll = ctx->d_coll; a.nspec = ctx->d_nspec; a.scal = ctx->d_scal;
    MG_CUDA(cudaMemsetAsync(ctx->d_scal, 0, 3 * sizeof(unsigned long long), ctx->stream));
    const unsigned grid = (unsigned)((ctx->n + 127) / 128);
    {
        MgTimed t(ctx, "stateq");
        if (ctx->n_lev <= 8) k_stateq<8><<<grid, 128, 0, ctx->stream>>>(a);
        else if (ctx->n_lev <= 24) k_stateq<24><<<grid, 128, 0, ctx->stream>>>(a);
        else k_stateq<64><<<grid, 128, 0, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    std::swap(ctx->d_pops, ctx->d_pops_new);
    return MG_OK;
}

// Statistical equilibrium from pops_old into pops_new with explicit buffers (no pointer
// swap), skipped when *active == 0; used by the batch graph.
int mg_launch_stateq_into(mg_ctx *ctx, const double *pops_old, double *pops_new, const int32_t *active) {
    StateqArgs a{};
    a.n = ctx->n; a.nlev = ctx->n_lev; a.L = ctx->n_lines; a.lc = ctx->d_lines;
    a.pops = pops_old; a.pops_new = pops_new; a.J = ctx->d_J; a.Lc = ctx->d_Lc; a.Jeff = ctx->d_Jeff;
    a.coll = ctx->d_coll; a.nspec = ctx->d_nspec; a.scal = ctx->d_scal; a.active = active;
    const unsigned grid = (unsigned)((ctx->n + 127) / 128);
    if (ctx->n_lev <= 8) k_stateq<8><<<grid, 128, 0, ctx->stream>>>(a);
    else if (ctx->n_lev <= 24) k_stateq<24><<<grid, 128, 0, ctx->stream>>>(a);
    else k_stateq<64><<<grid, 128, 0, ctx->stream>>>(a);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_push_history(mg_ctx *ctx) {
    const int64_t m = ctx->n * ctx->n_lev;
    int rc;
    for (auto &h : ctx->d_hist)
        if (!h && (rc = mg_alloc(ctx, &h, m))) return rc;
    double *t = ctx->d_hist[3];
    ctx->d_hist[3] = ctx->d_hist[2];
    ctx->d_hist[2] = ctx->d_hist[1];
    ctx->d_hist[1] = ctx->d_hist[0];
    ctx->d_hist[0] = t;
    k_push_history<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, ctx->n_lev, ctx->d_pops, ctx->d_nspec,
                                                                          ctx->d_hist[0]);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_ng(mg_ctx *ctx, int *accepted) {
    const int64_t m = ctx->n * ctx->n_lev;
    int rc;
    if (!ctx->d_ng_tmp && (rc = mg_alloc(ctx, &ctx->d_ng_tmp, m))) return rc;
    if (!ctx->d_ng_part && (rc = mg_alloc(ctx, &ctx->d_ng_part, 5 * kNgBlocks))) return rc;
    MG_CUDA(cudaMemsetAsync(ctx->d_scal + 3, 0, sizeof(unsigned long long), ctx->stream));
    {
        MgTimed t(ctx, "ng");
        k_ng_dots<<<kNgBlocks, kNgThreads, 0, ctx->stream>>>(m, ctx->d_hist[0], ctx->d_hist[1], ctx->d_hist[2],
                                                             ctx->d_hist[3], ctx->d_ng_part);
        k_ng_apply<<<kNgBlocks, kNgThreads, 0, ctx->stream>>>(m, ctx->n_lev, ctx->d_ng_part, kNgBlocks, ctx->d_hist[0],
                                                              ctx->d_hist[1], ctx->d_hist[2], ctx->d_nspec,
                                                              ctx->d_ng_tmp, ctx->d_scal + 3);
    }
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal + 3, ctx->d_scal + 3, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    *accepted = ctx->h_scal[3] == 0;
    if (*accepted)
        MG_CUDA(cudaMemcpyAsync(ctx->d_pops, ctx->d_ng_tmp, 8 * m, cudaMemcpyDeviceToDevice, ctx->stream));
    return MG_OK;
}
