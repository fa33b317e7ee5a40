// mg_update_populations_noalloc: the statistical-equilibrium update of
// mg_update_populations for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they update level populations:
// a host framework whose allocator already owns the GPU's memory and forbids other
// allocations, a loop that cannot afford the device-wide synchronisation an allocation
// may cause, or a process whose memory budget is fixed after start-up. This variant
// takes the old and new populations as caller-owned device buffers and keeps its only
// scratch -- per-block partial results of the convergence and fallback reductions -- in
// a file-scope static __device__ array. That array exists on every GPU that loads this
// library, from load until process exit.
//
// The collision rates are evaluated inside the kernel (same formulas and operation
// order as the context's collision-rate table), so the call depends only on the
// radiation field left by the last mg_formal_solve and on the model, species and
// quadrature already in the context.
#include <cmath>
#include <cstring>
#include "common.cuh"

using namespace mg;

namespace {

constexpr int kNaThreads = 128;
constexpr int64_t kNaMaxBlocks = 16384;                      // 512 KiB of partials
constexpr int64_t kNaMaxCells = kNaMaxBlocks * kNaThreads;   // 2,097,152 cells per call

// [kNaMaxBlocks][4]: max-change bits, fallback count, non-finite count, unused; then
// the final [4] result words. Every slot a call reads is written earlier in the same
// call, so nothing needs clearing; calls that overlap on the GPU race on this array.
static __device__ __align__(256) unsigned long long g_na_scratch[(kNaMaxBlocks + 1) * 4];

struct NaArgs {
    int64_t n;
    int nlev, L, nT;
    const LineConst *lc;
    const double *E, *g, *Tg, *K, *T, *ncoll, *nspec;
    const double *J, *Lc, *Jeff;
    const double *pops_old;
    double *pops_new;
    unsigned long long *scratch;
};

template <int MAXLEV>
__device__ bool na_gth(int n, double (&q)[MAXLEV][MAXLEV], double (&pi)[MAXLEV]) {
    double ex[MAXLEV];
    for (int k = n - 1; k >= 1; k--) {
        double s = 0.0;
        for (int j = 0; j < k; j++) s += q[k][j];
        ex[k] = s;
        if (!(s > 0.0)) return false;
        const double is = 1.0 / s;
        for (int i = 0; i < k; i++) {
            const double f = q[i][k] * is;
            if (f == 0.0) continue;
            for (int j = 0; j < k; j++) q[i][j] += f * q[k][j];
        }
    }
    pi[0] = 1.0;
    double tot = 1.0;
    for (int k = 1; k < n; k++) {
        double s = 0.0;
        for (int i = 0; i < k; i++) s += pi[i] * q[i][k];
        pi[k] = s / ex[k];
        tot += pi[k];
    }
    for (int k = 0; k < n; k++) pi[k] /= tot;
    return true;
}

template <int MAXLEV>
__device__ void na_rates(const NaArgs &a, int64_t c, bool plain, double (&q)[MAXLEV][MAXLEV]) {
    const int n = a.nlev;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) q[i][j] = 0.0;
    for (int l = 0; l < a.L; l++) {
        const LineConst k = a.lc[l];
        const double je = plain ? a.J[c * a.L + l] : a.Jeff[c * a.L + l];
        const double oml = plain ? 1.0 : a.Lc[c * a.L + l];
        q[k.up][k.lo] += k.A * oml + k.Bul * je;
        q[k.lo][k.up] += k.Blu * je;
    }
    const double Tc = a.T[c];
    int pr = 0;
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++, pr++) {
            const double *k = a.K + (size_t)pr * a.nT;
            double kd;
            if (a.nT == 1 || Tc <= a.Tg[0]) kd = k[0];
            else if (Tc >= a.Tg[a.nT - 1]) kd = k[a.nT - 1];
            else {
                int s = 0;
                while (a.Tg[s + 1] < Tc) s++;
                const double w = (Tc - a.Tg[s]) / (a.Tg[s + 1] - a.Tg[s]);
                kd = k[s] + w * (k[s + 1] - k[s]);
            }
            const double Cd = kd * a.ncoll[c];
            q[i][j] += Cd;
            q[j][i] += Cd * a.g[i] / a.g[j] * exp(-(a.E[i] - a.E[j]) / (kKB * Tc));
        }
}

template <int MAXLEV>
__global__ void __launch_bounds__(kNaThreads) k_stateq_noalloc(NaArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double change = 0.0;
    unsigned long long fb = 0, bad = 0;
    if (c < a.n) {
        const int n = a.nlev;
        double q[MAXLEV][MAXLEV], pi[MAXLEV];
        na_rates<MAXLEV>(a, c, false, q);
        bool ok = na_gth<MAXLEV>(n, q, pi);
        for (int i = 0; i < n && ok; i++) ok = isfinite(pi[i]) && pi[i] >= 0.0;
        if (!ok) {
            fb = 1;
            na_rates<MAXLEV>(a, c, true, q);
            ok = na_gth<MAXLEV>(n, q, pi);
            for (int i = 0; i < n && ok; i++) ok = isfinite(pi[i]) && pi[i] >= 0.0;
            if (!ok) bad = 1;
        }
        const double ns = a.nspec[c];
        for (int i = 0; i < n; i++) {
            const double nw = ns * pi[i];
            const double od = a.pops_old[c * n + i];
            a.pops_new[c * n + i] = nw;
            if (nw >= 1e-10 * ns) {
                const double d = fabs(nw - od) / nw;
                if (d > change) change = d;
            }
        }
        if (!isfinite(change)) change = INFINITY;
    }
    unsigned long long bits = __double_as_longlong(change);
    for (int d = 16; d; d >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, bits, d);
        bits = o > bits ? o : bits;
        fb += __shfl_down_sync(0xffffffffu, fb, d);
        bad += __shfl_down_sync(0xffffffffu, bad, d);
    }
    __shared__ unsigned long long w[kNaThreads / 32][3];
    if ((threadIdx.x & 31) == 0) {
        w[threadIdx.x >> 5][0] = bits;
        w[threadIdx.x >> 5][1] = fb;
        w[threadIdx.x >> 5][2] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0, f = 0, b = 0;
        for (int k = 0; k < kNaThreads / 32; k++) {
            m = w[k][0] > m ? w[k][0] : m;
            f += w[k][1];
            b += w[k][2];
        }
        unsigned long long *p = a.scratch + 4 * (size_t)blockIdx.x;
        p[0] = m; p[1] = f; p[2] = b; p[3] = 0;
    }
}

// Combines the per-block partials in block order and writes the result words.
__global__ void k_noalloc_finish(const unsigned long long *part, int64_t nblocks, unsigned long long *res) {
    __shared__ unsigned long long s[3][256];
    unsigned long long m = 0, f = 0, b = 0;
    for (int64_t k = threadIdx.x; k < nblocks; k += blockDim.x) {
        m = part[4 * k] > m ? part[4 * k] : m;
        f += part[4 * k + 1];
        b += part[4 * k + 2];
    }
    s[0][threadIdx.x] = m; s[1][threadIdx.x] = f; s[2][threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < (int)blockDim.x; t++) {
            m = s[0][t] > m ? s[0][t] : m;
            f += s[1][t];
            b += s[2][t];
        }
        res[0] = m; res[1] = f; res[2] = b; res[3] = 0;
    }
}

// Device address of g_na_scratch per device ordinal, looked up once per device.
constexpr int kNaMaxDevices = 64;
unsigned long long *g_na_ptr[kNaMaxDevices] = {nullptr};

}  // namespace

extern "C" int mg_update_populations_noalloc(mg_ctx *ctx, const double *d_pops_old, double *d_pops_new,
                                             double *max_rel_change, int64_t *n_fallback) {
    if (!ctx) return MG_ERR_ARG;
    if (!d_pops_old || !d_pops_new) return mg_fail(ctx, MG_ERR_ARG, "mg_update_populations_noalloc: null buffer");
    if (!ctx->have_rad || !ctx->d_Lc)
        return mg_fail(ctx, MG_ERR_STATE, "mg_update_populations_noalloc: run mg_formal_solve first");
    if (ctx->n > kNaMaxCells)
        return mg_fail(ctx, MG_ERR_CAPACITY,
                       "mg_update_populations_noalloc: at most 2097152 cells per call (static scratch of 512 KiB)");
    if (ctx->device < 0 || ctx->device >= kNaMaxDevices)
        return mg_fail(ctx, MG_ERR_ARG, "mg_update_populations_noalloc: device ordinal out of range");
    MG_CUDA(cudaSetDevice(ctx->device));
    if (!g_na_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return mg_cuda_check(ctx, e, "cudaGetSymbolAddress(g_na_scratch)");
        g_na_ptr[ctx->device] = static_cast<unsigned long long *>(p);
    }
    unsigned long long *scratch = g_na_ptr[ctx->device];
    NaArgs a{};
    a.n = ctx->n; a.nlev = ctx->n_lev; a.L = ctx->n_lines; a.nT = ctx->n_T;
    a.lc = ctx->d_lines; a.E = ctx->d_E; a.g = ctx->d_g; a.Tg = ctx->d_Tgrid; a.K = ctx->d_Kdown;
    a.T = ctx->d_T; a.ncoll = ctx->d_ncoll; a.nspec = ctx->d_nspec;
    a.J = ctx->d_J; a.Lc = ctx->d_Lc; a.Jeff = ctx->d_Jeff;
    a.pops_old = d_pops_old; a.pops_new = d_pops_new; a.scratch = scratch;
    const int64_t nb = (ctx->n + kNaThreads - 1) / kNaThreads;
    if (ctx->n_lev <= 8) k_stateq_noalloc<8><<<(unsigned)nb, kNaThreads, 0, ctx->stream>>>(a);
    else if (ctx->n_lev <= 24) k_stateq_noalloc<24><<<(unsigned)nb, kNaThreads, 0, ctx->stream>>>(a);
    else k_stateq_noalloc<64><<<(unsigned)nb, kNaThreads, 0, ctx->stream>>>(a);
    MG_CUDA(cudaGetLastError());
    unsigned long long *res = scratch + 4 * kNaMaxBlocks;
    k_noalloc_finish<<<1, 256, 0, ctx->stream>>>(scratch, nb, res);
    MG_CUDA(cudaGetLastError());
    unsigned long long h[4];
    MG_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    double ch;
    std::memcpy(&ch, &h[0], 8);
    if (max_rel_change) *max_rel_change = ch;
    if (n_fallback) *n_fallback = (int64_t)h[1];
    if (h[2]) return mg_fail(ctx, MG_ERR_NUMERIC, "statistical equilibrium: non-finite populations after fallback");
    return h[1] ? MG_WARN_NEG_POP_FALLBACK : MG_OK;
}
