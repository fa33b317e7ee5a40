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
// Everything that could allocate happens once, when the species is set
// (mg_noalloc_prepare, called by mg_set_species): loading this file's kernels and the
// static array on the device (lazy module loading allocates device memory for them),
// looking up the array's device address, and one warm-up launch of the kernel instance
// the species needs, so that its local-memory reservation (the rate matrix of up to 64
// levels lives in local memory) is made there. The update itself then allocates nothing.
//
// The collision rates are evaluated inside the kernel with the same device functions as
// the context's collision-rate table, and the rates and the GTH solve are those of the
// regular update (stateq_common.cuh), so the call depends only on the radiation field
// left by the last mg_formal_solve (or mg_set_radiation) and on the model and species.
#include <cmath>
#include <cstring>
#include <mutex>
#include "common.cuh"
#include "stateq_common.cuh"

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

// Rates of eq. 'ourALI' (or without the ALO when `plain`), the collision part evaluated
// in place from the tabulated coefficients.
template <int MAXLEV>
__device__ void na_rates(const NaArgs &a, int64_t c, bool plain, double (&q)[MAXLEV][MAXLEV]) {
    const int n = a.nlev;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) q[i][j] = 0.0;
    line_rates<MAXLEV>(a.L, a.lc, a.J, a.Lc, a.Jeff, c, plain, q);
    const double Tc = a.T[c];
    int pr = 0;
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++, pr++) {
            double Cd, Cu;
            collision_rates_pair(collision_k_down(a.K, pr, a.nT, a.Tg, Tc), a.ncoll[c], a.g[i], a.g[j], a.E[i],
                                 a.E[j], Tc, Cd, Cu);
            q[i][j] += Cd;
            q[j][i] += Cu;
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
        bool ok = gth_solve<MAXLEV>(n, q, pi) && valid_fractions<MAXLEV>(n, pi);
        if (!ok) {
            fb = 1;
            na_rates<MAXLEV>(a, c, true, q);
            ok = gth_solve<MAXLEV>(n, q, pi) && valid_fractions<MAXLEV>(n, pi);
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

// Device address of g_na_scratch per device ordinal, looked up once per device under a
// lock (two threads setting up contexts on the same device do not race on it).
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
unsigned long long *g_na_ptr[kNaMaxDevices] = {nullptr};

template <int MAXLEV>
int na_launch(const NaArgs &a, int64_t nb, cudaStream_t s) {
    k_stateq_noalloc<MAXLEV><<<(unsigned)nb, kNaThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

int na_dispatch(int nlev, const NaArgs &a, int64_t nb, cudaStream_t s) {
    if (nlev <= 8) return na_launch<8>(a, nb, s);
    if (nlev <= 24) return na_launch<24>(a, nb, s);
    return na_launch<64>(a, nb, s);
}

template <int MAXLEV>
cudaError_t na_attributes() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, k_stateq_noalloc<MAXLEV>);
}

}  // namespace

// Set-up for mg_update_populations_noalloc on the context's device and species (called
// by mg_set_species with the device current): the static scratch's device address, the
// kernels loaded, and one warm-up launch over no cells (one block that only writes its
// partial-result slot) so that the instance's local memory is reserved now. Failures are
// kept in the context and reported by the update; mg_set_species itself does not fail.
void mg_noalloc_prepare(mg_ctx *ctx) {
    ctx->na_ready = false;
    ctx->na_error.clear();
    if (ctx->device < 0 || ctx->device >= kNaMaxDevices) {
        ctx->na_error = "device ordinal out of range";
        return;
    }
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[ctx->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess) {
                ctx->na_error = std::string("cudaGetSymbolAddress(g_na_scratch): ") + cudaGetErrorString(e);
                return;
            }
            g_na_ptr[ctx->device] = static_cast<unsigned long long *>(p);
        }
        scratch = g_na_ptr[ctx->device];
    }
    cudaFuncAttributes fa;
    cudaError_t e = ctx->n_lev <= 8 ? na_attributes<8>() : (ctx->n_lev <= 24 ? na_attributes<24>() : na_attributes<64>());
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_noalloc_finish);
    if (e != cudaSuccess) {
        ctx->na_error = std::string("cudaFuncGetAttributes: ") + cudaGetErrorString(e);
        return;
    }
    NaArgs a{};
    a.n = 0;
    a.nlev = ctx->n_lev;
    a.scratch = scratch;
    if (na_dispatch(ctx->n_lev, a, 1, ctx->stream) != MG_OK) {
        ctx->na_error = "warm-up launch failed";
        return;
    }
    k_noalloc_finish<<<1, 256, 0, ctx->stream>>>(scratch, 1, scratch + 4 * kNaMaxBlocks);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ctx->na_error = std::string("warm-up: ") + cudaGetErrorString(e);
        return;
    }
    ctx->na_scratch = scratch;
    ctx->na_ready = true;
}

extern "C" int mg_update_populations_noalloc(mg_ctx *ctx, const double *d_pops_old, double *d_pops_new,
                                             double *max_rel_change, int64_t *n_fallback) {
    if (!ctx) return MG_ERR_ARG;
    if (!d_pops_old || !d_pops_new) return mg_fail(ctx, MG_ERR_ARG, "mg_update_populations_noalloc: null buffer");
    if (!ctx->have_rad || !ctx->d_Lc)
        return mg_fail(ctx, MG_ERR_STATE, "mg_update_populations_noalloc: run mg_formal_solve first");
    if (ctx->band_cur > 0)
        return mg_fail(ctx, MG_ERR_STATE,
                       "mg_update_populations_noalloc: needs the diagonal ALO (the band ALO's solver allocates)");
    if (ctx->n > kNaMaxCells)
        return mg_fail(ctx, MG_ERR_CAPACITY,
                       "mg_update_populations_noalloc: at most 2097152 cells per call (static scratch of 512 KiB)");
    if (!ctx->na_ready)
        return mg_fail(ctx, MG_ERR_CUDA, "mg_update_populations_noalloc: set-up at mg_set_species failed: " + ctx->na_error);
    MG_CUDA(cudaSetDevice(ctx->device));
    unsigned long long *scratch = ctx->na_scratch;
    NaArgs a{};
    a.n = ctx->n; a.nlev = ctx->n_lev; a.L = ctx->n_lines; a.nT = ctx->n_T;
    a.lc = ctx->d_lines; a.E = ctx->d_E; a.g = ctx->d_g; a.Tg = ctx->d_Tgrid; a.K = ctx->d_Kdown;
    a.T = ctx->d_T; a.ncoll = ctx->d_ncoll; a.nspec = ctx->d_nspec;
    a.J = ctx->d_J; a.Lc = ctx->d_Lc; a.Jeff = ctx->d_Jeff;
    a.pops_old = d_pops_old; a.pops_new = d_pops_new; a.scratch = scratch;
    const int64_t nb = (ctx->n + kNaThreads - 1) / kNaThreads;
    if (na_dispatch(ctx->n_lev, a, nb, ctx->stream) != MG_OK)
        return mg_cuda_check(ctx, cudaGetLastError(), "k_stateq_noalloc");
    unsigned long long *res = scratch + 4 * kNaMaxBlocks;
    k_noalloc_finish<<<1, 256, 0, ctx->stream>>>(scratch, nb, res);
    MG_CUDA(cudaGetLastError());
    // result words into the context's pinned words [5..7], the negative-opacity count of
    // the last formal solve into word [4] (as mg_update_populations reads it)
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal + 5, res, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal + 4, ctx->d_scal + 4, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    double ch;
    std::memcpy(&ch, &ctx->h_scal[5], 8);
    if (max_rel_change) *max_rel_change = ch;
    if (n_fallback) *n_fallback = (int64_t)ctx->h_scal[6];
    if (ctx->h_scal[7]) return mg_fail(ctx, MG_ERR_NUMERIC, "statistical equilibrium: non-finite populations after fallback");
    if (ctx->h_scal[6]) return MG_WARN_NEG_POP_FALLBACK;
    return ctx->h_scal[4] ? MG_WARN_NEG_OPACITY : MG_OK;
}
