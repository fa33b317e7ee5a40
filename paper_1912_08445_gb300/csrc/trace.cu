// K1: ray tracing by neighbour walk (Sec. 3.2) with the velocity-step rule (Sec. 3.1.1).
// This translation unit is compiled with --fmad=false: every floating-point decision of
// the walk (projections, distances, velocity steps) is reproducible bit for bit.
#include <cmath>
#include <algorithm>
#include "common.cuh"

using namespace mg;

namespace {

struct TraceArgs {
    int64_t n;
    int32_t R;
    int32_t geometry;
    const double *pos, *vel, *b, *dirs;
    const float4 *posf;                // (x, y, z, |x| + |y| + |z|) in FP32, for the filter
    const int64_t *nbr_off;
    const int32_t *nbr_idx;
    const uint8_t *bdy;
    double dshift_frac;
    int64_t max_steps;
    // count pass
    int32_t *len, *xlen;
    // fill pass
    const int64_t *ray_off;
    int32_t *cells, *xcum;
    double *ds, *vpar;
    int32_t *err;
    // cells of each half-ray recorded by the count pass: tmp[k * n R + t] for k < cap_tmp
    int32_t *tmp;
    int32_t cap_tmp;
};

// Points inserted between two consecutive points by the velocity-step rule: when the
// line-of-sight velocity changes by dv > f min(b_a, b_b), ceil(dv/(f min)) - 1 points.
__device__ __forceinline__ int32_t velocity_inserts(double va, double ba, double vb, double bb, double f) {
    double dv = fabs(vb - va);
    double wmin = ba < bb ? ba : bb;
    double lim = f * wmin;
    if (dv > lim) return (int32_t)ceil(dv / lim) - 1;
    return 0;
}

// Records one element of the half-ray. The count pass records only the cell (its count,
// and the first cells for the replay); the fill pass also the path length, the
// line-of-sight velocity and the expanded-point count of the velocity-step rule.
template <bool FILL>
__device__ __forceinline__ bool emit(const TraceArgs &a, int64_t base, int32_t &len, int32_t &x, int32_t cell,
                                     double ds, double vp, double &va, double &ba) {
    if (len >= a.max_steps) return false;
    if (FILL) {
        double bb = a.b[cell];
        int32_t ns = velocity_inserts(va, ba, vp, bb, a.dshift_frac);
        x += ns + 1;
        a.cells[base + len] = cell;
        a.xcum[base + len] = x;
        a.ds[base + len] = ds;
        a.vpar[base + len] = vp;
        va = vp;
        ba = bb;
    } else if (a.tmp && len < a.cap_tmp) {
        a.tmp[(int64_t)len * a.n * a.R + base] = cell;   // base = thread index in the count pass
    }
    len++;
    return true;
}

// 3D point cloud: from the current cell, the neighbour with a strictly larger projection
// on the ray that lies closest to the ray (ties: smaller squared distance, smaller
// projection, smaller index); stop after a boundary cell or at a dead end.
//
// The decisions are those of the FP64 expressions below, bit for bit, but most of them
// are taken in FP32 (64x the FP64 rate on this GPU) with a rigorous error bound, and FP64
// is evaluated only where the bound cannot decide:
// - a candidate is valid when s > s_cur: the FP32 projection decides unless it lies
//   within its error bound of s_cur, where the FP64 projection decides;
// - the FP32 squared distance of every valid candidate comes with an interval
//   [lo, hi] that contains the FP64 value; the FP64 winner's lo is at most the smallest
//   hi, so every valid candidate with lo <= min hi is evaluated in FP64 and the winner
//   is chosen among those with the exact tie-breaks. (A non-finite bound leaves the
//   candidate to FP64.)
// The bounds follow from |fl32(a) - a| <= u|a| (u = 2^-24) for the conversions of the
// positions and the direction and for each FP32 operation; they are doubled for margin.
struct Cand32 {
    bool valid;
    float lo, hi;   // interval of the FP64 squared distance
};

__device__ __forceinline__ double proj64(const TraceArgs &a, int64_t c, double xo0, double xo1, double xo2,
                                         double n0, double n1, double n2) {
    const double dx = a.pos[3 * c] - xo0;
    const double dy = a.pos[3 * c + 1] - xo1;
    const double dz = a.pos[3 * c + 2] - xo2;
    return dx * n0 + dy * n1 + dz * n2;
}

__device__ __forceinline__ Cand32 classify32(const TraceArgs &a, int64_t c, const float4 po, float n0f, float n1f,
                                             float n2f, float scf, double s_cur, double xo0, double xo1,
                                             double xo2, double n0, double n1, double n2) {
    constexpr float k2u = 1.2e-7f;   // 2u with margin
    const float4 pc = a.posf[c];
    const float dx = pc.x - po.x, dy = pc.y - po.y, dz = pc.z - po.z;
    const float D = fabsf(dx) + fabsf(dy) + fabsf(dz);
    const float P = pc.w + po.w;
    const float sf = dx * n0f + dy * n1f + dz * n2f;
    const float Es = k2u * (P + 6.0f * D);   // |sf - s64|
    const float diff = sf - scf;
    const float margin = Es + k2u * (fabsf(scf) + fabsf(diff));
    Cand32 r;
    if (diff > margin) r.valid = true;
    else if (diff < -margin) r.valid = false;
    else r.valid = proj64(a, c, xo0, xo1, xo2, n0, n1, n2) > s_cur;   // inconclusive in FP32
    const float px = dx - sf * n0f, py = dy - sf * n1f, pz = dz - sf * n2f;
    const float d2 = px * px + py * py + pz * pz;
    const float Ep = 2.0f * (Es + 0.6e-7f * (P + 4.0f * D + 3.0f * fabsf(sf)));   // |px - px64| and so on
    const float Ed = 1.1f * (2.0f * Ep * (fabsf(px) + fabsf(py) + fabsf(pz)) + 9.0f * Ep * Ep + k2u * 2.0f * d2);
    r.lo = d2 - Ed;
    r.hi = d2 + Ed;
    return r;
}

template <bool FILL>
__device__ void walk_3d(const TraceArgs &a, int64_t o, int r, int64_t base, int32_t &len, int32_t &x,
                        bool &dead, bool &overflow) {
    const double n0 = a.dirs[3 * r], n1 = a.dirs[3 * r + 1], n2 = a.dirs[3 * r + 2];
    const double xo0 = a.pos[3 * o], xo1 = a.pos[3 * o + 1], xo2 = a.pos[3 * o + 2];
    const double vo0 = a.vel[3 * o], vo1 = a.vel[3 * o + 1], vo2 = a.vel[3 * o + 2];
    const float n0f = (float)n0, n1f = (float)n1, n2f = (float)n2;
    const float4 po = a.posf[o];
    int64_t cur = o;
    double s_cur = 0.0;
    double va = 0.0, ba = a.b[o];
    len = 0;
    x = 0;
    dead = false;
    overflow = false;
    for (;;) {
        const float scf = (float)s_cur;
        const int64_t e0 = a.nbr_off[cur], e1 = a.nbr_off[cur + 1];
        // pass 1: validity, the smallest upper bound of a valid candidate's distance, and
        // the two smallest lower bounds
        float minhi = INFINITY, lo1 = INFINITY, lo2 = INFINITY;
        int64_t c1 = -1;
        bool full = false;   // a bound that is not finite leaves the choice to pass 2
        for (int64_t e = e0; e < e1; e++) {
            const int64_t c = a.nbr_idx[e];
            const Cand32 k = classify32(a, c, po, n0f, n1f, n2f, scf, s_cur, xo0, xo1, xo2, n0, n1, n2);
            if (!k.valid) continue;
            if (!(k.lo <= k.hi) || !(fabsf(k.hi) < INFINITY)) full = true;
            minhi = fminf(minhi, k.hi);
            if (k.lo < lo1) {
                lo2 = lo1;
                lo1 = k.lo;
                c1 = c;
            } else if (k.lo < lo2) {
                lo2 = k.lo;
            }
        }
        int64_t best = -1;
        double bs = 0.0, bd2 = 0.0;
        // Only the candidate with the smallest lower bound reaches min hi: it is the
        // closest, and only its FP64 projection is needed.
        const bool unique = c1 >= 0 && !full && lo2 > minhi;
        if (unique) {
            best = c1;
            bs = proj64(a, c1, xo0, xo1, xo2, n0, n1, n2);
        }
        // pass 2: FP64 for every valid candidate that may be the closest
        for (int64_t e = unique ? e1 : e0; e < e1; e++) {
            const int64_t c = a.nbr_idx[e];
            const Cand32 k = classify32(a, c, po, n0f, n1f, n2f, scf, s_cur, xo0, xo1, xo2, n0, n1, n2);
            if (!k.valid || k.lo > minhi) continue;
            const double dx = a.pos[3 * c] - xo0;
            const double dy = a.pos[3 * c + 1] - xo1;
            const double dz = a.pos[3 * c + 2] - xo2;
            const double s = dx * n0 + dy * n1 + dz * n2;
            const double px = dx - s * n0, py = dy - s * n1, pz = dz - s * n2;
            const double d2 = px * px + py * py + pz * pz;
            const bool better = (best < 0) || (d2 < bd2) || (d2 == bd2 && s < bs) || (d2 == bd2 && s == bs && c < best);
            if (better) { best = c; bs = s; bd2 = d2; }
        }
        if (best < 0) { dead = true; return; }
        const double vp = FILL ? n0 * (a.vel[3 * best] - vo0) + n1 * (a.vel[3 * best + 1] - vo1) +
                                     n2 * (a.vel[3 * best + 2] - vo2)
                               : 0.0;
        if (!emit<FILL>(a, base, len, x, (int32_t)best, bs - s_cur, vp, va, ba)) { overflow = true; return; }
        s_cur = bs;
        cur = best;
        if (a.bdy[best]) return;
    }
}

// Fill pass of a half-ray whose cells the count pass recorded: the same projections,
// path lengths, line-of-sight velocities and velocity steps as the walk, without the
// neighbour search.
__device__ void replay_3d(const TraceArgs &a, int64_t o, int r, int64_t t, int64_t base, int32_t n_cells) {
    const double n0 = a.dirs[3 * r], n1 = a.dirs[3 * r + 1], n2 = a.dirs[3 * r + 2];
    const double xo0 = a.pos[3 * o], xo1 = a.pos[3 * o + 1], xo2 = a.pos[3 * o + 2];
    const double vo0 = a.vel[3 * o], vo1 = a.vel[3 * o + 1], vo2 = a.vel[3 * o + 2];
    double s_cur = 0.0, va = 0.0, ba = a.b[o];
    int32_t len = 0, x = 0;
    for (int32_t k = 0; k < n_cells; k++) {
        const int64_t c = a.tmp[(int64_t)k * a.n * a.R + t];
        const double dx = a.pos[3 * c] - xo0;
        const double dy = a.pos[3 * c + 1] - xo1;
        const double dz = a.pos[3 * c + 2] - xo2;
        const double s = dx * n0 + dy * n1 + dz * n2;
        const double vp = n0 * (a.vel[3 * c] - vo0) + n1 * (a.vel[3 * c + 1] - vo1) + n2 * (a.vel[3 * c + 2] - vo2);
        emit<true>(a, base, len, x, (int32_t)c, s - s_cur, vp, va, ba);
        s_cur = s;
    }
}

// Spherically symmetric shells on +z: crossings of the ray with sphere j at
// s = -r_o mu +- sqrt(r_j^2 - r_o^2 (1 - mu^2)), in increasing s; an empty core below the
// first radius carries no path length; a first radius of 0 is a centre point.
template <bool FILL>
__device__ void walk_sph1d(const TraceArgs &a, int64_t o, int r, int64_t base, int32_t &len, int32_t &x,
                           bool &overflow) {
    const double mu = a.dirs[3 * r + 2];
    const double ro = a.pos[3 * o + 2];
    const double p2 = ro * ro * (1.0 - mu * mu);
    const double vro = a.vel[3 * o + 2];
    const int64_t N = a.n;
    const double r0 = a.pos[2];
    double va = 0.0, ba = a.b[o];
    double s_prev = 0.0;
    len = 0;
    x = 0;
    overflow = false;
    int64_t j = o;
    bool through_core = false;
    const bool inward = (mu < 0.0 && ro > 0.0);
    if (inward) {
        for (j = o - 1; j >= 0; j--) {
            const double rj = a.pos[3 * j + 2];
            const double q = rj * rj - p2;
            if (rj == 0.0 && p2 == 0.0) {
                const double s = -ro * mu;
                if (!emit<FILL>(a, base, len, x, (int32_t)j, s - s_prev, -vro * mu, va, ba)) { overflow = true; return; }
                s_prev = s;
                j--;
                break;
            }
            if (!(q > 0.0) || rj == 0.0) break;
            const double s = -ro * mu - sqrt(q);
            const double vp = a.vel[3 * j + 2] * (ro * mu + s) / rj - vro * mu;
            if (!emit<FILL>(a, base, len, x, (int32_t)j, s - s_prev, vp, va, ba)) { overflow = true; return; }
            s_prev = s;
        }
        if (j < 0 && r0 > 0.0) through_core = true;
        j = j + 1;
        if (j == 0 && r0 == 0.0) j = 1;
    }
    const int64_t jstart = inward ? j : o + 1;
    for (int64_t k = jstart; k < N; k++) {
        const double rk = a.pos[3 * k + 2];
        const double q = rk * rk - p2;
        if (q < 0.0) continue;
        const double s = -ro * mu + sqrt(q);
        const bool core_chord = through_core && k == jstart;
        if (!(s > s_prev) && !core_chord) continue;
        const double dsv = core_chord ? 0.0 : s - s_prev;
        const double vp = (rk > 0.0 ? a.vel[3 * k + 2] * (ro * mu + s) / rk : 0.0) - vro * mu;
        if (!emit<FILL>(a, base, len, x, (int32_t)k, dsv, vp, va, ba)) { overflow = true; return; }
        s_prev = s;
    }
}

// One thread per (origin, direction); consecutive threads take consecutive origins of the
// same direction so that neighbouring walks share cache lines.
template <bool FILL>
__global__ void k_trace(TraceArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n * a.R) return;
    const int r = (int)(t / a.n);
    const int64_t o = t - (int64_t)r * a.n;
    const int64_t ray = o * a.R + r;
    const int64_t base = FILL ? a.ray_off[ray] : t;
    int32_t len = 0, x = 0;
    bool dead = false, overflow = false;
    if (FILL && a.tmp && a.geometry == MG_GEOM_3D) {
        const int32_t n_cells = a.len[ray];
        if (n_cells <= a.cap_tmp) {
            replay_3d(a, o, r, t, base, n_cells);
            return;
        }
    }
    if (a.geometry == MG_GEOM_SPHERICAL_1D) walk_sph1d<FILL>(a, o, r, base, len, x, overflow);
    else walk_3d<FILL>(a, o, r, base, len, x, dead, overflow);
    if (overflow) atomicOr(a.err, 1);
    if (!FILL) {
        a.len[ray] = len;
        a.xlen[ray] = dead ? -1 : 0;   // dead-end flag; the expanded lengths come from the fill pass
    }
}

// ---------------------------------------------------------------- exclusive scan
// Exclusive prefix sum of int32 counts into int64 offsets, in three passes: per-block
// sums, a single-block scan of the block sums, then per-block scans with their offsets.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += y;
    }
    return v;
}

__device__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        s = warp_incl_scan(s);
        wsum[lane] = s;
    }
    __syncthreads();
    int64_t off = w ? wsum[w - 1] : 0;
    if (total) *total = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return off + inc - v;
}

__global__ void k_scan_blocks(const int32_t *cnt, int64_t m, int64_t *bsum) {
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = i < m ? cnt[i] : 0;
    int64_t tot;
    block_excl_scan(v, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t *bsum, int64_t nb) {
    // single block: sequential chunks of kScanBlock
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanBlock) {
        int64_t i = c0 + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, &tot);
        if (i < nb) bsum[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const int32_t *cnt, int64_t m, const int64_t *bsum, int64_t *out) {
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = i < m ? cnt[i] : 0;
    int64_t ex = block_excl_scan(v, nullptr);
    if (i < m) out[i] = bsum[blockIdx.x] + ex;
    if (i == m - 1) out[m] = bsum[blockIdx.x] + ex + v;
}

// Expanded length of every half-ray from the filled store (xcum of its last cell), with
// the count pass's dead-end flag kept as the sign (-x - 1).
__global__ void k_xlen(int64_t nr, const int64_t *__restrict__ ray_off, const int32_t *__restrict__ len,
                       const int32_t *__restrict__ xcum, int32_t *__restrict__ xlen) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr) return;
    const int32_t x = len[t] ? xcum[ray_off[t] + len[t] - 1] : 0;
    xlen[t] = xlen[t] < 0 ? -x - 1 : x;
}

// ---------------------------------------------------------------- statistics
__global__ void k_ray_stats(int64_t n, int R, int P, const int32_t *pf, const int32_t *pb, const int32_t *len,
                            int32_t *xlen, unsigned long long *st) {
    // st: [0] elements, [1] expanded, [2] max pair length, [3] dead ends
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long el = 0, ex = 0, mx = 0, dead = 0;
    if (t < n * R) {
        int32_t xv = xlen[t];
        if (xv < 0) { dead = 1; xv = -xv - 1; xlen[t] = xv; }
        el = (unsigned long long)len[t];
        ex = (unsigned long long)xv;
    }
    __syncthreads();
    if (t < n * P) {
        const int64_t o = t / P;
        const int p = (int)(t - o * P);
        int32_t a = xlen[o * R + pf[p]], b = xlen[o * R + pb[p]];
        a = a < 0 ? -a - 1 : a;
        b = b < 0 ? -b - 1 : b;
        mx = (unsigned long long)(a + b + 1);
    }
    for (int d = 16; d; d >>= 1) {
        el += __shfl_down_sync(0xffffffffu, el, d);
        ex += __shfl_down_sync(0xffffffffu, ex, d);
        dead += __shfl_down_sync(0xffffffffu, dead, d);
        unsigned long long m2 = __shfl_down_sync(0xffffffffu, mx, d);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st[0], el);
        atomicAdd(&st[1], ex);
        atomicMax(&st[2], mx);
        atomicAdd(&st[3], dead);
    }
}

__global__ void k_to_float(const double *a, float *b, int64_t m) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = (float)a[i];
}

}  // namespace

int mg_scan_counts(mg_ctx *ctx, const int32_t *d_cnt, int64_t m, int64_t *d_out) {
    int64_t nb = (m + kScanBlock - 1) / kScanBlock;
    int64_t *bsum = nullptr;
    int rc;
    if ((rc = mg_alloc(ctx, &bsum, nb))) return rc;
    k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(d_cnt, m, bsum);
    k_scan_sums<<<1, kScanBlock, 0, ctx->stream>>>(bsum, nb);
    k_scan_apply<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(d_cnt, m, bsum, d_out);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    cudaFree(bsum);
    if (e != cudaSuccess) return mg_cuda_check(ctx, e, "scan");
    return MG_OK;
}

__global__ void k_posf(int64_t n, const double *__restrict__ pos, float4 *__restrict__ posf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = (float)pos[3 * i], y = (float)pos[3 * i + 1], z = (float)pos[3 * i + 2];
    posf[i] = make_float4(x, y, z, fabsf(x) + fabsf(y) + fabsf(z));
}

// Temporaries of one trace, freed on every return (cudaFree waits for the kernels that
// may still use them).
struct TraceScratch {
    int32_t *len = nullptr, *xlen = nullptr, *tmp = nullptr;
    float4 *posf = nullptr;
    ~TraceScratch() {
        cudaFree(len);
        cudaFree(xlen);
        cudaFree(tmp);
        cudaFree(posf);
    }
};

int mg_launch_trace(mg_ctx *ctx) {
    const int64_t nr = ctx->n * ctx->R;
    int rc;
    TraceScratch sc;
    if ((rc = mg_alloc(ctx, &sc.len, nr)) || (rc = mg_alloc(ctx, &sc.xlen, nr))) return rc;
    int32_t *const d_len = sc.len, *const d_xlen = sc.xlen;
    if ((rc = mg_alloc(ctx, &ctx->d_ray_off, nr + 1))) return rc;
    MG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), ctx->stream));
    TraceArgs a{};
    a.n = ctx->n; a.R = ctx->R; a.geometry = ctx->geometry;
    a.pos = ctx->d_pos; a.vel = ctx->d_vel; a.b = ctx->d_b; a.dirs = ctx->d_dirs;
    a.nbr_off = ctx->d_nbr_off; a.nbr_idx = ctx->d_nbr_idx; a.bdy = ctx->d_bdy;
    a.dshift_frac = ctx->opt.dshift_frac; a.max_steps = ctx->opt.max_steps;
    a.len = d_len; a.xlen = d_xlen; a.err = ctx->d_err;
    if (ctx->geometry == MG_GEOM_3D) {
        if ((rc = mg_alloc(ctx, &sc.posf, ctx->n))) return rc;
        k_posf<<<(unsigned)((ctx->n + 255) / 256), 256, 0, ctx->stream>>>(ctx->n, ctx->d_pos, sc.posf);
    }
    a.posf = sc.posf;
    // Record up to cap_tmp cells per half-ray in the count pass, in scratch of at most
    // 32 GiB and a quarter of the free device memory (freed after tracing; half-rays with
    // more cells, or all of them without scratch, are walked again by the fill pass).
    int32_t *&d_tmp = sc.tmp;
    int32_t cap_tmp = 128;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    const double budget = std::min(32.0 * (1 << 30), 0.25 * (double)free_b);
    while (cap_tmp > 0 && (double)nr * cap_tmp * 4.0 > budget) cap_tmp /= 2;
    if (ctx->geometry == MG_GEOM_3D && cap_tmp > 0 && cudaMalloc(&d_tmp, (size_t)nr * cap_tmp * 4) != cudaSuccess) {
        cudaGetLastError();
        d_tmp = nullptr;
    }
    a.tmp = d_tmp;
    a.cap_tmp = d_tmp ? cap_tmp : 0;
    const int bs = 128;
    const unsigned grid = (unsigned)((nr + bs - 1) / bs);
    {
        MgTimed t(ctx, "trace_count");
        k_trace<false><<<grid, bs, 0, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    if ((rc = mg_scan_counts(ctx, d_len, nr, ctx->d_ray_off))) return rc;
    int64_t total = 0;
    int32_t kerr = 0;
    MG_CUDA(cudaMemcpy(&total, ctx->d_ray_off + nr, 8, cudaMemcpyDeviceToHost));
    MG_CUDA(cudaMemcpy(&kerr, ctx->d_err, 4, cudaMemcpyDeviceToHost));
    if (kerr) {
        return mg_fail(ctx, MG_ERR_CAPACITY, "ray tracing: a half-ray exceeded max_steps");
    }
    if ((rc = mg_alloc(ctx, &ctx->d_cells, total)) || (rc = mg_alloc(ctx, &ctx->d_xcum, total)) ||
        (rc = mg_alloc(ctx, &ctx->d_ds, total)) || (rc = mg_alloc(ctx, &ctx->d_vpar, total)) ||
        (rc = mg_alloc(ctx, &ctx->d_dsf, total)) || (rc = mg_alloc(ctx, &ctx->d_vparf, total)))
        return rc;
    a.ray_off = ctx->d_ray_off; a.cells = ctx->d_cells; a.xcum = ctx->d_xcum; a.ds = ctx->d_ds; a.vpar = ctx->d_vpar;
    {
        MgTimed t(ctx, "trace_fill");
        k_trace<true><<<grid, bs, 0, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    if (total) {
        k_to_float<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_ds, ctx->d_dsf, total);
        k_to_float<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_vpar, ctx->d_vparf, total);
    }
    k_xlen<<<(unsigned)((nr + 255) / 256), 256, 0, ctx->stream>>>(nr, ctx->d_ray_off, d_len, ctx->d_xcum, d_xlen);
    MG_CUDA(cudaMemsetAsync(ctx->d_scal, 0, 4 * sizeof(unsigned long long), ctx->stream));
    const int64_t np = std::max<int64_t>(nr, ctx->n * ctx->P);
    k_ray_stats<<<(unsigned)((np + 255) / 256), 256, 0, ctx->stream>>>(ctx->n, ctx->R, ctx->P, ctx->d_pf, ctx->d_pb,
                                                                          d_len, d_xlen, ctx->d_scal);
    MG_CUDA(cudaGetLastError());
    unsigned long long st[4];
    MG_CUDA(cudaMemcpyAsync(st, ctx->d_scal, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->n_elements = (int64_t)st[0];
    ctx->n_expanded = (int64_t)st[1];
    ctx->max_pair_len = (int64_t)st[2];
    ctx->n_dead = (int64_t)st[3];
    ctx->traced = true;
    return MG_OK;
}
