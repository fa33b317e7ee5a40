// Statistical equilibrium with the band-diagonal approximate Lambda operator (Sec. 3.4,
// eq. 'ALO', 'ourALI'), its validity check and bandwidth reduction (Sec. 6.1).
//
// With an ALO of bandwidth B > 0 the rate equations of a cell o contain, for every line
// l = (u -> lo), the upper population at the band points of each half-ray: a point
// interpolates its line data between cells ca and cb with weight w on cb, and enters
// with coefficient A_ul M[o][l][r][j] (M from the FP64 formal solve). The share on the
// origin itself lowers the factor 1 - L of the spontaneous rate; the other cells couple
// the equations of all cells into one sparse linear system
//     B_o n_o + sum_c K(o, c) n_c = (0, ..., 0, n_spec(o)),
// where B_o is the cell's rate generator with its last row replaced by the
// normalisation sum_i n_i = n_spec, and K(o, c) adds A_ul M w n_u(c) to the balance of u
// and subtracts it from that of lo (none in the normalisation row). The unknowns are
// scaled by the old populations (n = s x, s = max(n_old, 1e-20 n_spec)) and the system is
// preconditioned by its block diagonal:
//     x + S^-1 B^-1 K S x = S^-1 B^-1 rhs,
// solved by restarted GMRES (classical Gram-Schmidt applied twice; dot products as
// fixed-order block sums, so reruns are bitwise identical). The solution is valid when
// every population is finite and non-negative; otherwise (or when GMRES does not reach
// its tolerance) the system is solved again with bandwidth B - 1, down to the diagonal
// ALO of stateq.cu, whose own check re-solves single cells without the ALO.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "stateq_common.cuh"

using namespace mg;

namespace {

constexpr int kBT = 128;          // threads per block of the per-cell kernels
constexpr int kDotBlocks = 304;   // 2 x 152 SMs: partial sums of the dot products
constexpr int kDotThreads = 128;
constexpr int kMaxKrylov = 30;    // restart length
constexpr int kMaxRestarts = 12;
constexpr double kTol = 1e-13;    // relative residual of the preconditioned system

// Cells and weight behind band slot j (0-based) of half-ray (o, r): the (j+1)-th
// expanded point from the origin lies in element e, sub-point (j + 1 - x0) of its
// ns + 1 points, interpolating between the element's predecessor and its cell with
// weight (j + 1 - x0)/(ns + 1) on the cell (the staging's expression).
__global__ void k_band_geometry(int64_t n, int R, int B, const int64_t *ray_off, const int32_t *cells,
                                const int32_t *xcum, int2 *cc, double *w) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    const int64_t o = t / R;
    const int64_t off = ray_off[t];
    const int len = (int)(ray_off[t + 1] - off);
    for (int j = 0; j < B; j++) {
        int2 c2 = make_int2(-1, -1);
        double ww = 0.0;
        int x0 = 0;
        int32_t prev = (int32_t)o;
        for (int e = 0; e < len; e++) {
            const int x1 = xcum[off + e];
            if (j < x1) {
                c2 = make_int2(prev, cells[off + e]);
                ww = (double)(j + 1 - x0) / (double)(x1 - x0);
                break;
            }
            x0 = x1;
            prev = cells[off + e];
        }
        cc[t * B + j] = c2;
        w[t * B + j] = ww;
    }
}

struct BandArgs {
    int64_t n;
    int nlev, L, R, B, Bs, Bg;        // bandwidth of this solve; strides of M and of the geometry
    const LineConst *lc;
    const double *oml, *Jeff;         // 1 - L [n][L], J_eff of bandwidth B [n][L]
    const double *M;                  // [n][L][R][Bs]
    const int2 *bc;                   // [n][R][Bg] cells (ca, cb)
    const double *bw;                 // [n][R][Bg] weight on cb
    const double *coll;               // [n][npairs][2]
    const double *nspec;
    const double *pops_old;           // [n][nlev]
    double *lu;                       // [n][nlev][nlev]
    int32_t *piv;                     // [n][nlev]
    double *s;                        // [n][nlev] scale of the unknowns
    double *z;                        // [n][nlev] preconditioned right-hand side
    unsigned long long *flag;         // singular blocks
};

// LU decomposition with partial pivoting in place (row-major n x n), pivot rows in p.
template <int MAXLEV>
__device__ bool lu_decompose(int n, double (&a)[MAXLEV][MAXLEV], int32_t (&p)[MAXLEV]) {
    for (int c = 0; c < n; c++) {
        int pr = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(a[r][c]) > fabs(a[pr][c])) pr = r;
        p[c] = pr;
        if (!(a[pr][c] != 0.0) || !isfinite(a[pr][c])) return false;
        if (pr != c)
            for (int k = 0; k < n; k++) { const double t = a[c][k]; a[c][k] = a[pr][k]; a[pr][k] = t; }
        const double id = 1.0 / a[c][c];
        for (int r = c + 1; r < n; r++) {
            const double f = a[r][c] * id;
            a[r][c] = f;
            if (f != 0.0)
                for (int k = c + 1; k < n; k++) a[r][k] -= f * a[c][k];
        }
    }
    return true;
}

// Solves with a stored factorisation (global memory, row-major) in place.
template <int MAXLEV>
__device__ void lu_solve_stored(int n, const double *a, const int32_t *p, double (&b)[MAXLEV]) {
    for (int c = 0; c < n; c++) {
        const int pr = p[c];
        if (pr != c) { const double t = b[c]; b[c] = b[pr]; b[pr] = t; }
        for (int r = c + 1; r < n; r++) b[r] -= a[r * n + c] * b[c];
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= a[r * n + k] * b[k];
        b[r] = s / a[r * n + r];
    }
}

// Per cell: the block B_o (rates with 1 - L lowered by the band points on the origin
// itself), its LU factors, the scale and the preconditioned right-hand side.
template <int MAXLEV>
__global__ void __launch_bounds__(kBT) k_band_setup(BandArgs a) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.n) return;
    const int n = a.nlev;
    // generator G_ij = rate j -> i, G_jj = -sum_i rate j -> i, assembled rate by rate
    double g[MAXLEV][MAXLEV];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) g[i][j] = 0.0;
    auto rate = [&](int from, int to, double v) {
        g[to][from] += v;
        g[from][from] -= v;
    };
    for (int l = 0; l < a.L; l++) {
        double self = 0.0;
        const double *Ml = a.M + ((size_t)o * a.L + l) * a.R * a.Bs;
        for (int r = 0; r < a.R; r++)
            for (int j = 0; j < a.B; j++) {
                const int2 c2 = a.bc[((size_t)o * a.R + r) * a.Bg + j];
                const double w = a.bw[((size_t)o * a.R + r) * a.Bg + j];
                const double m = Ml[r * a.Bs + j];
                if (c2.y == (int32_t)o) self += w * m;
                if (c2.x == (int32_t)o) self += (1.0 - w) * m;
            }
        const LineConst k = a.lc[l];
        const double je = a.Jeff[o * a.L + l];
        rate(k.up, k.lo, k.A * (a.oml[o * a.L + l] - self) + k.Bul * je);
        rate(k.lo, k.up, k.Blu * je);
    }
    const int npairs = n * (n - 1) / 2;
    const double *cr = a.coll + (size_t)o * npairs * 2;
    int pr = 0;
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++, pr++) {
            rate(i, j, cr[2 * pr]);
            rate(j, i, cr[2 * pr + 1]);
        }
    for (int j = 0; j < n; j++) g[n - 1][j] = 1.0;   // normalisation row
    int32_t p[MAXLEV];
    const bool ok = lu_decompose<MAXLEV>(n, g, p);
    double *lu = a.lu + (size_t)o * n * n;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) lu[i * n + j] = g[i][j];
        a.piv[o * n + i] = p[i];
    }
    const double ns = a.nspec[o];
    double b[MAXLEV];
    for (int i = 0; i < n; i++) b[i] = 0.0;
    b[n - 1] = ns;
    if (ok) lu_solve_stored<MAXLEV>(n, lu, a.piv + o * n, b);
    else atomicAdd(a.flag, 1ull);
    for (int i = 0; i < n; i++) {
        const double sc = fmax(a.pops_old[o * n + i], 1e-20 * ns);
        a.s[o * n + i] = sc;
        a.z[o * n + i] = ok ? b[i] / sc : 0.0;
    }
}

// y = x + S^-1 B^-1 K S x, the preconditioned operator on the scaled unknowns.
template <int MAXLEV>
__global__ void __launch_bounds__(kBT) k_band_apply(BandArgs a, const double *x, double *y) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.n) return;
    const int n = a.nlev;
    double t[MAXLEV];
    for (int i = 0; i < n; i++) t[i] = 0.0;
    for (int r = 0; r < a.R; r++)
        for (int j = 0; j < a.B; j++) {
            const int2 c2 = a.bc[((size_t)o * a.R + r) * a.Bg + j];
            if (c2.y < 0) continue;
            const double w = a.bw[((size_t)o * a.R + r) * a.Bg + j];
            for (int l = 0; l < a.L; l++) {
                const LineConst k = a.lc[l];
                const double m = k.A * a.M[(((size_t)o * a.L + l) * a.R + r) * a.Bs + j];
                double v = 0.0;
                if (c2.y != (int32_t)o) v += w * a.s[(size_t)c2.y * n + k.up] * x[(size_t)c2.y * n + k.up];
                if (c2.x != (int32_t)o && w != 1.0)
                    v += (1.0 - w) * a.s[(size_t)c2.x * n + k.up] * x[(size_t)c2.x * n + k.up];
                t[k.up] += m * v;
                t[k.lo] -= m * v;
            }
        }
    t[n - 1] = 0.0;
    lu_solve_stored<MAXLEV>(n, a.lu + (size_t)o * n * n, a.piv + o * n, t);
    for (int i = 0; i < n; i++) y[o * n + i] = x[o * n + i] + t[i] / a.s[o * n + i];
}

// ---------------------------------------------------------------- GMRES vector kernels
// Partial dot products <V_c, w> for c < ncols (V: ncols vectors of length N, stride N),
// one partial per block, summed in block order by k_dots_finish.
__global__ void __launch_bounds__(kDotThreads) k_dots(int64_t N, int ncols, const double *V, const double *w,
                                                        double *part) {
    __shared__ double sh[kMaxKrylov + 1][kDotThreads];
    double acc[kMaxKrylov + 1];
    for (int c = 0; c <= kMaxKrylov; c++) acc[c] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll 1
        for (int c = 0; c < ncols; c++) acc[c] += V[(size_t)c * N + i] * wi;
    }
    for (int c = 0; c < ncols; c++) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = kDotThreads / 2; h; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < ncols; c++) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        __syncthreads();
    }
    if ((int)threadIdx.x < ncols) part[(size_t)blockIdx.x * (kMaxKrylov + 1) + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_dots_finish(int ncols, const double *part, double *out) {
    const int c = threadIdx.x;
    if (c >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < kDotBlocks; b++) s += part[(size_t)b * (kMaxKrylov + 1) + c];
    out[c] = s;
}

// w -= sum_c V_c h_c (h on the device).
__global__ void k_sub_combination(int64_t N, int ncols, const double *V, const double *h, double *w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int c = 0; c < ncols; c++) s -= V[(size_t)c * N + i] * h[c];
        w[i] = s;
    }
}

// x += sum_c V_c y_c (y on the device).
__global__ void k_add_combination(int64_t N, int ncols, const double *V, const double *y, double *x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int c = 0; c < ncols; c++) s += V[(size_t)c * N + i] * y[c];
        x[i] = s;
    }
}

__global__ void k_scale_into(int64_t N, const double *w, const double *f, double *v) {
    const double inv = 1.0 / *f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = w[i] * inv;
}

__global__ void k_residual(int64_t N, const double *z, const double *y, double *r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = z[i] - y[i];
}

// n = s x into pops_new; validity (finite, non-negative) and the convergence measure as
// in k_stateq: [0] max change bits, [1] invalid cells.
__global__ void k_band_finish(int64_t ncell, int nlev, const double *x, const double *s, const double *nspec,
                              const double *pops_old, double *pops_new, unsigned long long *scal) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double change = 0.0;
    unsigned long long bad = 0;
    if (c < ncell) {
        const double ns = nspec[c];
        for (int i = 0; i < nlev; i++) {
            const double nw = s[c * nlev + i] * x[c * nlev + i];
            pops_new[c * nlev + i] = nw;
            if (!(isfinite(nw) && nw >= 0.0)) bad = 1;
            if (nw >= 1e-10 * ns) {
                const double d = fabs(nw - pops_old[c * nlev + i]) / nw;
                if (d > change) change = d;
            }
        }
        if (!isfinite(change)) change = INFINITY;
    }
    unsigned long long bits = __double_as_longlong(change);
    for (int d = 16; d; d >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, bits, d);
        bits = o > bits ? o : bits;
        bad += __shfl_down_sync(0xffffffffu, bad, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&scal[0], bits);
        if (bad) atomicAdd(&scal[1], bad);
    }
}

template <int MAXLEV>
int band_kernels_setup(const BandArgs &a, cudaStream_t st) {
    k_band_setup<MAXLEV><<<(unsigned)((a.n + kBT - 1) / kBT), kBT, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
template <int MAXLEV>
int band_kernels_apply(const BandArgs &a, const double *x, double *y, cudaStream_t st) {
    k_band_apply<MAXLEV><<<(unsigned)((a.n + kBT - 1) / kBT), kBT, 0, st>>>(a, x, y);
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

}  // namespace

void mg_band_free(mg_ctx *ctx) {
    mg_free(ctx->d_Jeffb); mg_free(ctx->d_Mb); mg_free(ctx->d_bcells); mg_free(ctx->d_bw); mg_free(ctx->d_blu);
    mg_free(ctx->d_bpiv); mg_free(ctx->d_bs); mg_free(ctx->d_bz); mg_free(ctx->d_bx); mg_free(ctx->d_bw2);
    mg_free(ctx->d_bV); mg_free(ctx->d_bpart); mg_free(ctx->d_bh);
    ctx->band_cap_n = 0;
    ctx->band_geo_ready = false;
}

// Buffers of the band solve, sized for the context's bandwidth (opt.alo_band).
int mg_band_alloc(mg_ctx *ctx) {
    const int Bm = ctx->opt.alo_band;
    const int64_t n = ctx->n, N = n * ctx->n_lev;
    int rc;
    if (ctx->band_cap_n == n && ctx->band_cap_lev == ctx->n_lev && ctx->band_cap_L == ctx->n_lines &&
        ctx->band_cap_R == ctx->R && ctx->d_Mb)
        return MG_OK;
    if ((rc = mg_alloc(ctx, &ctx->d_Jeffb, (size_t)Bm * n * ctx->n_lines)) ||
        (rc = mg_alloc(ctx, &ctx->d_Mb, (size_t)n * ctx->n_lines * ctx->R * Bm)) ||
        (rc = mg_alloc(ctx, &ctx->d_bcells, (size_t)n * ctx->R * Bm)) ||
        (rc = mg_alloc(ctx, &ctx->d_bw, (size_t)n * ctx->R * Bm)) ||
        (rc = mg_alloc(ctx, &ctx->d_blu, (size_t)n * ctx->n_lev * ctx->n_lev)) ||
        (rc = mg_alloc(ctx, &ctx->d_bpiv, (size_t)N)) || (rc = mg_alloc(ctx, &ctx->d_bs, (size_t)N)) ||
        (rc = mg_alloc(ctx, &ctx->d_bz, (size_t)N)) || (rc = mg_alloc(ctx, &ctx->d_bx, (size_t)N)) ||
        (rc = mg_alloc(ctx, &ctx->d_bw2, (size_t)N)) ||
        (rc = mg_alloc(ctx, &ctx->d_bV, (size_t)(kMaxKrylov + 1) * N)) ||
        (rc = mg_alloc(ctx, &ctx->d_bpart, (size_t)kDotBlocks * (kMaxKrylov + 1))) ||
        (rc = mg_alloc(ctx, &ctx->d_bh, (size_t)2 * (kMaxKrylov + 2))))
        return rc;
    ctx->band_cap_n = n;
    ctx->band_cap_lev = ctx->n_lev;
    ctx->band_cap_L = ctx->n_lines;
    ctx->band_cap_R = ctx->R;
    ctx->band_geo_ready = false;
    return MG_OK;
}

// Geometry of the band points of every half-ray (once per traced ray store).
int mg_band_geometry(mg_ctx *ctx) {
    if (ctx->band_geo_ready) return MG_OK;
    const int Bm = ctx->opt.alo_band;
    const int64_t m = ctx->n * ctx->R;
    k_band_geometry<<<(unsigned)((m + 127) / 128), 128, 0, ctx->stream>>>(ctx->n, ctx->R, Bm, ctx->d_ray_off,
                                                                        ctx->d_cells, ctx->d_xcum,
                                                                        ctx->d_bcells, ctx->d_bw);
    MG_CUDA(cudaGetLastError());
    ctx->band_geo_ready = true;
    return MG_OK;
}

// One solve of the coupled rate equations with bandwidth B (<= the bandwidth of the last
// formal solve) into ctx->d_pops_new. *valid: every population finite and non-negative
// and GMRES converged; *iters: GMRES iterations; scal words [0] max change, [1] invalid.
static int band_solve(mg_ctx *ctx, int B, bool *valid, int *iters) {
    const int64_t n = ctx->n, N = n * ctx->n_lev;
    const int lev = ctx->n_lev;
    cudaStream_t st = ctx->stream;
    BandArgs a{};
    if (B > ctx->band_solved) return mg_fail(ctx, MG_ERR_STATE, "band ALO: the formal solve has fewer band terms");
    a.n = n; a.nlev = lev; a.L = ctx->n_lines; a.R = ctx->R; a.B = B;
    a.Bs = ctx->band_solved;       // stride of the coupling terms of the last formal solve
    a.Bg = ctx->opt.alo_band;      // stride of the geometry table
    a.lc = ctx->d_lines; a.oml = ctx->d_Lc;
    a.Jeff = ctx->d_Jeffb + (size_t)(B - 1) * n * ctx->n_lines;
    a.M = ctx->d_Mb; a.bc = ctx->d_bcells; a.bw = ctx->d_bw;
    a.coll = ctx->d_coll; a.nspec = ctx->d_nspec; a.pops_old = ctx->d_pops;
    a.lu = ctx->d_blu; a.piv = ctx->d_bpiv; a.s = ctx->d_bs; a.z = ctx->d_bz; a.flag = ctx->d_scal + 5;
    MG_CUDA(cudaMemsetAsync(ctx->d_scal + 5, 0, sizeof(unsigned long long), st));
    int rc = lev <= 8 ? band_kernels_setup<8>(a, st) : (lev <= 24 ? band_kernels_setup<24>(a, st) : band_kernels_setup<64>(a, st));
    if (rc) return mg_cuda_check(ctx, cudaGetLastError(), "k_band_setup");
    auto apply = [&](const double *x, double *y) {
        return lev <= 8 ? band_kernels_apply<8>(a, x, y, st)
                        : (lev <= 24 ? band_kernels_apply<24>(a, x, y, st) : band_kernels_apply<64>(a, x, y, st));
    };
    const unsigned vb = 4 * 152, vt = 256;   // grid of the vector kernels
    double *x = ctx->d_bx, *w = ctx->d_bw2, *V = ctx->d_bV, *z = ctx->d_bz, *dh = ctx->d_bh;
    // ||z||
    k_dots<<<kDotBlocks, kDotThreads, 0, st>>>(N, 1, z, z, ctx->d_bpart);
    k_dots_finish<<<1, 32, 0, st>>>(1, ctx->d_bpart, dh);
    double h_host[kMaxKrylov + 2];
    MG_CUDA(cudaMemcpyAsync(h_host, dh, 8, cudaMemcpyDeviceToHost, st));
    unsigned long long sing = 0;
    MG_CUDA(cudaMemcpyAsync(&sing, ctx->d_scal + 5, 8, cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    const double znorm = std::sqrt(h_host[0]);
    *iters = 0;
    *valid = false;
    if (sing || !(znorm > 0.0) || !std::isfinite(znorm)) return MG_OK;
    MG_CUDA(cudaMemcpyAsync(x, z, 8 * (size_t)N, cudaMemcpyDeviceToDevice, st));   // block-Jacobi start
    bool conv = false;
    std::vector<double> H((size_t)(kMaxKrylov + 1) * kMaxKrylov), cs(kMaxKrylov), sn(kMaxKrylov), gg(kMaxKrylov + 1);
    for (int restart = 0; restart < kMaxRestarts && !conv; restart++) {
        // r = z - A x into V_0 (unnormalised), beta = ||r||
        if ((rc = apply(x, w))) return mg_cuda_check(ctx, cudaGetLastError(), "k_band_apply");
        k_residual<<<vb, vt, 0, st>>>(N, z, w, w);
        k_dots<<<kDotBlocks, kDotThreads, 0, st>>>(N, 1, w, w, ctx->d_bpart);
        k_dots_finish<<<1, 32, 0, st>>>(1, ctx->d_bpart, dh);
        MG_CUDA(cudaMemcpyAsync(h_host, dh, 8, cudaMemcpyDeviceToHost, st));
        MG_CUDA(cudaStreamSynchronize(st));
        const double beta = std::sqrt(h_host[0]);
        if (!std::isfinite(beta)) return MG_OK;
        if (beta <= kTol * znorm) { conv = true; break; }
        // V_0 = r / beta (the divisor is read from a device word)
        h_host[0] = beta;
        MG_CUDA(cudaMemcpyAsync(dh + kMaxKrylov + 1, h_host, 8, cudaMemcpyHostToDevice, st));
        k_scale_into<<<vb, vt, 0, st>>>(N, w, dh + kMaxKrylov + 1, V);
        std::fill(gg.begin(), gg.end(), 0.0);
        gg[0] = beta;
        int k = 0;
        for (; k < kMaxKrylov; k++) {
            double *vk = V + (size_t)k * N;
            if ((rc = apply(vk, w))) return mg_cuda_check(ctx, cudaGetLastError(), "k_band_apply");
            // classical Gram-Schmidt, twice
            double hc[kMaxKrylov + 1];
            for (int c = 0; c <= k; c++) hc[c] = 0.0;
            for (int pass = 0; pass < 2; pass++) {
                k_dots<<<kDotBlocks, kDotThreads, 0, st>>>(N, k + 1, V, w, ctx->d_bpart);
                k_dots_finish<<<1, 32, 0, st>>>(k + 1, ctx->d_bpart, dh);
                k_sub_combination<<<vb, vt, 0, st>>>(N, k + 1, V, dh, w);
                MG_CUDA(cudaMemcpyAsync(h_host, dh, 8 * (size_t)(k + 1), cudaMemcpyDeviceToHost, st));
                MG_CUDA(cudaStreamSynchronize(st));
                for (int c = 0; c <= k; c++) hc[c] += h_host[c];
            }
            k_dots<<<kDotBlocks, kDotThreads, 0, st>>>(N, 1, w, w, ctx->d_bpart);
            k_dots_finish<<<1, 32, 0, st>>>(1, ctx->d_bpart, dh);
            MG_CUDA(cudaMemcpyAsync(h_host, dh, 8, cudaMemcpyDeviceToHost, st));
            MG_CUDA(cudaStreamSynchronize(st));
            const double hn = std::sqrt(h_host[0]);
            (*iters)++;
            // Givens rotations of the new Hessenberg column
            for (int c = 0; c < k; c++) {
                const double t = cs[c] * hc[c] + sn[c] * hc[c + 1];
                hc[c + 1] = -sn[c] * hc[c] + cs[c] * hc[c + 1];
                hc[c] = t;
            }
            const double den = std::hypot(hc[k], hn);
            cs[k] = den > 0.0 ? hc[k] / den : 1.0;
            sn[k] = den > 0.0 ? hn / den : 0.0;
            hc[k] = den;
            gg[k + 1] = -sn[k] * gg[k];
            gg[k] = cs[k] * gg[k];
            for (int c = 0; c <= k; c++) H[(size_t)c * kMaxKrylov + k] = hc[c];
            const bool done = std::fabs(gg[k + 1]) <= kTol * znorm || !(hn > 0.0);
            if (!done && k + 1 < kMaxKrylov) {
                h_host[0] = hn;
                MG_CUDA(cudaMemcpyAsync(dh + kMaxKrylov + 1, h_host, 8, cudaMemcpyHostToDevice, st));
                k_scale_into<<<vb, vt, 0, st>>>(N, w, dh + kMaxKrylov + 1, V + (size_t)(k + 1) * N);
            }
            if (done) { k++; break; }
        }
        // y from the triangular system, x += V y
        std::vector<double> y(k, 0.0);
        for (int r = k - 1; r >= 0; r--) {
            double s = gg[r];
            for (int c = r + 1; c < k; c++) s -= H[(size_t)r * kMaxKrylov + c] * y[c];
            y[r] = s / H[(size_t)r * kMaxKrylov + r];
        }
        MG_CUDA(cudaMemcpyAsync(dh, y.data(), 8 * (size_t)k, cudaMemcpyHostToDevice, st));
        k_add_combination<<<vb, vt, 0, st>>>(N, k, V, dh, x);
        MG_CUDA(cudaGetLastError());
        MG_CUDA(cudaStreamSynchronize(st));   // y is a host buffer
    }
    if (!conv) {   // the last restart's residual, checked directly
        if ((rc = apply(x, w))) return mg_cuda_check(ctx, cudaGetLastError(), "k_band_apply");
        k_residual<<<vb, vt, 0, st>>>(N, z, w, w);
        k_dots<<<kDotBlocks, kDotThreads, 0, st>>>(N, 1, w, w, ctx->d_bpart);
        k_dots_finish<<<1, 32, 0, st>>>(1, ctx->d_bpart, dh);
        MG_CUDA(cudaMemcpyAsync(h_host, dh, 8, cudaMemcpyDeviceToHost, st));
        MG_CUDA(cudaStreamSynchronize(st));
        conv = std::sqrt(h_host[0]) <= kTol * znorm;
    }
    MG_CUDA(cudaMemsetAsync(ctx->d_scal, 0, 2 * sizeof(unsigned long long), st));
    k_band_finish<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, lev, x, ctx->d_bs, ctx->d_nspec, ctx->d_pops,
                                                               ctx->d_pops_new, ctx->d_scal);
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    *valid = conv && ctx->h_scal[1] == 0;
    return MG_OK;
}

// Statistical equilibrium with the band ALO of bandwidth ctx->band_cur (> 0): solved with
// that bandwidth, and again with smaller ones while the solution is not valid; the
// bandwidth in use keeps the reduction. Bandwidth 0 is the diagonal ALO of stateq.cu
// (mg_launch_stateq). On success the new populations are in d_pops (swapped) and
// *max_change, the fallback count and the bandwidth used are set.
int mg_band_update(mg_ctx *ctx, double *max_change, int64_t *n_fallback, int *band_used) {
    int rc;
    for (int B = ctx->band_cur; B > 0; B--) {
        bool valid = false;
        int iters = 0;
        if ((rc = band_solve(ctx, B, &valid, &iters))) return rc;
        ctx->band_gmres_iters += iters;
        if (valid) {
            double ch;
            std::memcpy(&ch, &ctx->h_scal[0], 8);
            *max_change = ch;
            *n_fallback = 0;
            *band_used = B;
            ctx->band_cur = B;
            std::swap(ctx->d_pops, ctx->d_pops_new);
            return MG_OK;
        }
    }
    ctx->band_cur = 0;
    *band_used = 0;
    if ((rc = mg_launch_stateq(ctx))) return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    double ch;
    std::memcpy(&ch, &ctx->h_scal[0], 8);
    *max_change = ch;
    *n_fallback = (int64_t)ctx->h_scal[1];
    if (ctx->h_scal[2]) return mg_fail(ctx, MG_ERR_NUMERIC, "statistical equilibrium: non-finite populations after fallback");
    return MG_OK;
}
