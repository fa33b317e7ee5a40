// C ABI entry points, host-side set-up (directions, quadrature, species tables) and the
// ALI driver of libmagritte_gb300.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include "common.cuh"

using namespace mg;

int mg_fail(const mg_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int mg_cuda_check(const mg_ctx *ctx, cudaError_t e, const char *what) {
    return mg_fail(ctx, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

MgTimed::MgTimed(mg_ctx *c, const char *name) : ctx(c), idx(-1) {
    if (!ctx->opt.profile) return;
    for (size_t i = 0; i < ctx->timers.size(); i++)
        if (ctx->timers[i].name == name) idx = (int)i;
    if (idx < 0) {
        ctx->timers.push_back(KernelTimer{name, 0.0, 0});
        idx = (int)ctx->timers.size() - 1;
    }
    cudaEventRecord(ctx->ev0, ctx->stream);
}

MgTimed::~MgTimed() {
    if (idx < 0) return;
    cudaEventRecord(ctx->ev1, ctx->stream);
    cudaEventSynchronize(ctx->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->timers[idx].ms += ms;
    ctx->timers[idx].launches += 1;
}

// ------------------------------------------------------------------ options / lifetime
extern "C" void mg_default_options(mg_options *o) {
    std::memset(o, 0, sizeof(*o));
    o->precision = MG_FP64;
    o->device = 0;
    o->tol = 1e-6;
    o->max_iter = 300;
    o->ng_period = 4;
    o->dshift_frac = 1.0 / 3.0;
    o->chi_min = 1e-30;
    o->dtau_min = 1e-30;
    o->T_cmb = 2.725;
    o->line_cut = 7.5;
    o->max_steps = 100000;
    o->profile = 0;
    o->spectrum = 0;
    o->tau_fp64 = 0.0;
    o->alo_band = 0;
}

extern "C" int mg_create(mg_ctx **out, const mg_options *opt) {
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    mg_ctx *ctx = new mg_ctx();
    if (opt) ctx->opt = *opt;
    else mg_default_options(&ctx->opt);
    const mg_options &o = ctx->opt;
    if ((o.precision != MG_FP64 && o.precision != MG_MIXED) || !(o.tol > 0) || o.max_iter < 1 ||
        o.ng_period < 0 || !(o.dshift_frac > 0) || !(o.chi_min > 0) || !(o.dtau_min > 0) ||
        !(o.T_cmb > 0) || !(o.line_cut > 0) || o.max_steps < 1 || !(o.tau_fp64 >= 0) ||
        (o.tau_fp64 > 0 && o.tau_fp64 <= 1) || o.alo_band < 0 || o.alo_band > 2 ||
        (o.alo_band > 0 && o.precision != MG_FP64)) {
        delete ctx;
        return MG_ERR_ARG;
    }
    ctx->device = o.device;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_scal, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_scal, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_err, sizeof(int32_t));
    if (e != cudaSuccess) {
        mg_destroy(ctx);
        return MG_ERR_CUDA;
    }
    ctx->stream = ctx->own_stream;
    ctx->band_cur = o.alo_band;
    cudaMemset(ctx->d_scal, 0, 8 * sizeof(unsigned long long));
    *out = ctx;
    return MG_OK;
}

static void free_rays(mg_ctx *ctx) {
    mg_free(ctx->d_ray_off); mg_free(ctx->d_cells); mg_free(ctx->d_xcum); mg_free(ctx->d_ds);
    mg_free(ctx->d_vpar); mg_free(ctx->d_dsf); mg_free(ctx->d_vparf);
    ctx->traced = false;
    ctx->band_geo_ready = false;
}

static void drop_state(mg_ctx *ctx) {
    mg_free(ctx->d_pops); mg_free(ctx->d_pops_new); mg_free(ctx->d_line); mg_free(ctx->d_linef);
    mg_free(ctx->d_J); mg_free(ctx->d_L); mg_free(ctx->d_Jeff); mg_free(ctx->d_Lc); mg_free(ctx->d_Jnu);
    for (auto &h : ctx->d_hist) mg_free(h);
    mg_free(ctx->d_ng_tmp); mg_free(ctx->d_ng_part); mg_free(ctx->d_promo);
    // image buffers are sized by the point and line counts
    mg_free(ctx->d_img); mg_free(ctx->d_imgxy); mg_free(ctx->d_imgov); mg_free(ctx->d_imglf);
    ctx->img_cap = 0;
    mg_band_free(ctx);
    ctx->band_solved = 0;
    // scattering buffers are sized by the point, line and bin counts: set them again
    mg_free(ctx->d_chisca); mg_free(ctx->d_Jsca); mg_free(ctx->d_Jsca_new); mg_free(ctx->d_scaw);
    ctx->sca_on = false;
}

extern "C" int mg_destroy(mg_ctx *ctx) {
    if (!ctx) return MG_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_rays(ctx);
    mg_free(ctx->d_pos); mg_free(ctx->d_vel); mg_free(ctx->d_nbr_off); mg_free(ctx->d_nbr_idx);
    mg_free(ctx->d_bdy); mg_free(ctx->d_ncoll); mg_free(ctx->d_T); mg_free(ctx->d_nspec);
    mg_free(ctx->d_b); mg_free(ctx->d_bf); mg_free(ctx->d_lines); mg_free(ctx->d_lconst); mg_free(ctx->d_E); mg_free(ctx->d_g);
    mg_free(ctx->d_Tgrid); mg_free(ctx->d_Kdown); mg_free(ctx->d_coll); mg_free(ctx->d_ovl_off);
    mg_free(ctx->d_ovl); mg_free(ctx->d_dirs); mg_free(ctx->d_pf); mg_free(ctx->d_pb);
    mg_free(ctx->d_roots); mg_free(ctx->d_weights); mg_free(ctx->d_pops); mg_free(ctx->d_pops_new);
    for (auto &h : ctx->d_hist) mg_free(h);
    mg_free(ctx->d_ng_tmp); mg_free(ctx->d_ng_part); mg_free(ctx->d_promo);
    mg_free(ctx->d_line); mg_free(ctx->d_linef); mg_free(ctx->d_J); mg_free(ctx->d_L);
    mg_free(ctx->d_Jeff); mg_free(ctx->d_Lc); mg_free(ctx->d_Jnu); mg_free(ctx->d_scal);
    mg_free(ctx->d_err);
    mg_free(ctx->d_uch); mg_free(ctx->d_img); mg_free(ctx->d_imgxy); mg_free(ctx->d_imgov); mg_free(ctx->d_imglf);
    mg_band_free(ctx);
    mg_free(ctx->d_chisca); mg_free(ctx->d_Jsca); mg_free(ctx->d_Jsca_new); mg_free(ctx->d_scaw);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return MG_OK;
}

extern "C" const char *mg_last_error(const mg_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int mg_set_stream(mg_ctx *ctx, void *stream) {
    if (!ctx) return MG_ERR_ARG;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return MG_OK;
}

// ------------------------------------------------------------------ mesh and model
static int upload(mg_ctx *ctx, void *dst, const void *src, size_t bytes) {
    MG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return MG_OK;
}

extern "C" int mg_set_mesh(mg_ctx *ctx, int64_t n, const double *pos, const double *vel,
                           const int64_t *nbr_off, const int32_t *nbr_idx, const uint8_t *is_bdy,
                           int32_t geometry) {
    if (!ctx) return MG_ERR_ARG;
    if (n < 1 || n > INT32_MAX || !pos || !vel || !nbr_off || !nbr_idx || !is_bdy)
        return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: bad size or null pointer");
    if (geometry != MG_GEOM_3D && geometry != MG_GEOM_SPHERICAL_1D)
        return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: unknown geometry");
    if (nbr_off[0] != 0) return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: nbr_off[0] != 0");
    for (int64_t i = 0; i < n; i++)
        if (nbr_off[i + 1] < nbr_off[i]) return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: nbr_off not monotone");
    int64_t E = nbr_off[n];
    for (int64_t e = 0; e < E; e++)
        if (nbr_idx[e] < 0 || nbr_idx[e] >= n) return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: neighbour index out of range");
    if (geometry == MG_GEOM_SPHERICAL_1D) {
        for (int64_t i = 0; i < n; i++) {
            if (pos[3 * i] != 0.0 || pos[3 * i + 1] != 0.0 || pos[3 * i + 2] < 0.0 ||
                (i > 0 && !(pos[3 * i + 2] > pos[3 * (i - 1) + 2])))
                return mg_fail(ctx, MG_ERR_ARG, "mg_set_mesh: spherical shells must lie on +z with increasing radius");
        }
    }
    cudaSetDevice(ctx->device);
    free_rays(ctx);
    drop_state(ctx);
    ctx->n = n;
    ctx->geometry = geometry;
    ctx->n_edges = E;
    ctx->vmax = 0.0;
    for (int64_t i = 0; i < n; i++)
        ctx->vmax = std::max(ctx->vmax, std::sqrt(vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                                                  vel[3 * i + 2] * vel[3 * i + 2]));
    {   // longest path through the model
        double lo[3] = {pos[0], pos[1], pos[2]}, hi[3] = {pos[0], pos[1], pos[2]}, rmax = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < 3; k++) {
                lo[k] = std::min(lo[k], pos[3 * i + k]);
                hi[k] = std::max(hi[k], pos[3 * i + k]);
                rmax = std::max(rmax, std::fabs(pos[3 * i + k]));
            }
        ctx->extent = geometry == MG_GEOM_SPHERICAL_1D
                          ? 2.0 * rmax
                          : std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                      (hi[2] - lo[2]) * (hi[2] - lo[2]));
    }
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_pos, 3 * n)) || (rc = mg_alloc(ctx, &ctx->d_vel, 3 * n)) ||
        (rc = mg_alloc(ctx, &ctx->d_nbr_off, n + 1)) || (rc = mg_alloc(ctx, &ctx->d_nbr_idx, E)) ||
        (rc = mg_alloc(ctx, &ctx->d_bdy, n)))
        return rc;
    if ((rc = upload(ctx, ctx->d_pos, pos, 24 * n)) || (rc = upload(ctx, ctx->d_vel, vel, 24 * n)) ||
        (rc = upload(ctx, ctx->d_nbr_off, nbr_off, 8 * (n + 1))) ||
        (rc = upload(ctx, ctx->d_nbr_idx, nbr_idx, 4 * E)) || (rc = upload(ctx, ctx->d_bdy, is_bdy, n)))
        return rc;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->have_mesh = true;
    ctx->have_model = false;
    ctx->have_pops = false;
    ctx->have_rad = false;
    ctx->coll_ready = false;
    return MG_OK;
}

// Velocity width b = sqrt(2 k T / m + v_turb^2). The expression and its operation order
// are fixed because the ray tracer compares velocity steps against it exactly.
static double width_of(double T, double vt, double mass) {
    double vth2 = 2.0 * kKB * T / mass;
    return std::sqrt(vth2 + vt * vt);
}

static int refresh_widths(mg_ctx *ctx) {
    if (!ctx->have_model || !ctx->have_species) return MG_OK;
    std::vector<double> b(ctx->n);
    std::vector<float> bf(ctx->n);
    ctx->bmax = 0.0;
    for (int64_t i = 0; i < ctx->n; i++) {
        b[i] = width_of(ctx->h_T[i], ctx->h_vturb[i], ctx->mass);
        ctx->bmax = std::max(ctx->bmax, b[i]);
        bf[i] = (float)b[i];
    }
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_b, ctx->n)) || (rc = mg_alloc(ctx, &ctx->d_bf, ctx->n))) return rc;
    if ((rc = upload(ctx, ctx->d_b, b.data(), 8 * ctx->n)) || (rc = upload(ctx, ctx->d_bf, bf.data(), 4 * ctx->n)))
        return rc;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

extern "C" int mg_set_model(mg_ctx *ctx, const double *n_coll, const double *T, const double *v_turb,
                            const double *n_species) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_mesh) return mg_fail(ctx, MG_ERR_STATE, "mg_set_model: set the mesh first");
    if (!n_coll || !T || !v_turb || !n_species) return mg_fail(ctx, MG_ERR_ARG, "mg_set_model: null pointer");
    int64_t n = ctx->n;
    for (int64_t i = 0; i < n; i++)
        if (!(T[i] > 0) || !(n_coll[i] >= 0) || !(v_turb[i] >= 0) || !(n_species[i] > 0))
            return mg_fail(ctx, MG_ERR_ARG, "mg_set_model: T and n_species must be > 0, n_coll and v_turb >= 0");
    cudaSetDevice(ctx->device);
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_ncoll, n)) || (rc = mg_alloc(ctx, &ctx->d_T, n)) ||
        (rc = mg_alloc(ctx, &ctx->d_nspec, n)))
        return rc;
    if ((rc = upload(ctx, ctx->d_ncoll, n_coll, 8 * n)) || (rc = upload(ctx, ctx->d_T, T, 8 * n)) ||
        (rc = upload(ctx, ctx->d_nspec, n_species, 8 * n)))
        return rc;
    ctx->h_T.assign(T, T + n);
    ctx->h_vturb.assign(v_turb, v_turb + n);
    ctx->have_model = true;
    ctx->coll_ready = false;
    free_rays(ctx);   // widths change the velocity-step insertions
    return refresh_widths(ctx);
}

static void build_overlaps(mg_ctx *ctx) {
    // Lines l' whose profile can reach a bin of line l anywhere in the model: within
    // the largest Doppler offset (twice the largest speed), the outermost root times
    // the widest width, and line_cut widths of l'.
    int L = ctx->n_lines;
    ctx->h_ovl_off.assign(L + 1, 0);
    ctx->h_ovl.clear();
    double bmax = 0.0;
    for (int64_t i = 0; i < (int64_t)ctx->h_T.size(); i++)
        bmax = std::max(bmax, width_of(ctx->h_T[i], ctx->h_vturb[i], ctx->mass));
    double rmax = 0.0;
    for (double r : ctx->h_roots) rmax = std::max(rmax, std::fabs(r));
    if (rmax == 0.0) rmax = 15.0;
    double vmax = 1e6;   // generous bound on |v| differences (1000 km/s) when unknown
    for (int l = 0; l < L; l++) {
        for (int l2 = 0; l2 < L; l2++) {
            double nl = ctx->h_lines[l].nu, n2 = ctx->h_lines[l2].nu;
            double reach = (nl * (rmax * bmax + 2.0 * vmax) + ctx->opt.line_cut * n2 * bmax) / kC;
            if (l2 == l || std::fabs(nl - n2) <= 1.01 * reach) {
                Overlap o;
                o.dnl = kC * (nl - n2) / n2;
                o.rat = nl / n2;
                o.inv_nu2 = 1.0 / n2;
                o.l2 = l2;
                o.pad = 0;
                if (l2 == l) {   // own line first
                    ctx->h_ovl.insert(ctx->h_ovl.begin() + ctx->h_ovl_off[l], o);
                } else {
                    ctx->h_ovl.push_back(o);
                }
            }
        }
        ctx->h_ovl_off[l + 1] = (int32_t)ctx->h_ovl.size();
    }
}

static int upload_overlaps(mg_ctx *ctx) {
    build_overlaps(ctx);
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_ovl_off, ctx->h_ovl_off.size())) ||
        (rc = mg_alloc(ctx, &ctx->d_ovl, ctx->h_ovl.size())))
        return rc;
    if ((rc = upload(ctx, ctx->d_ovl_off, ctx->h_ovl_off.data(), 4 * ctx->h_ovl_off.size())) ||
        (rc = upload(ctx, ctx->d_ovl, ctx->h_ovl.data(), sizeof(Overlap) * ctx->h_ovl.size())))
        return rc;
    return MG_OK;
}

extern "C" int mg_set_species(mg_ctx *ctx, int32_t n_lev, const double *E, const double *g, double mass,
                              int32_t n_lines, const int32_t *up, const int32_t *lo, const double *A,
                              int32_t n_T, const double *T_grid, const double *K_down) {
    if (!ctx) return MG_ERR_ARG;
    if (n_lev < 2 || n_lev > kMaxLev || n_lines < 1 || n_T < 1 || !(mass > 0) || !E || !g || !up || !lo ||
        !A || !T_grid || !K_down)
        return mg_fail(ctx, MG_ERR_ARG, "mg_set_species: bad sizes or null pointer");
    for (int i = 0; i < n_lev; i++)
        if (!(g[i] > 0)) return mg_fail(ctx, MG_ERR_ARG, "mg_set_species: g must be > 0");
    for (int l = 0; l < n_lines; l++) {
        if (up[l] < 0 || up[l] >= n_lev || lo[l] < 0 || lo[l] >= n_lev || !(E[up[l]] > E[lo[l]]) || !(A[l] >= 0))
            return mg_fail(ctx, MG_ERR_ARG, "mg_set_species: line levels must satisfy E[up] > E[lo], A >= 0");
    }
    for (int t = 1; t < n_T; t++)
        if (!(T_grid[t] > T_grid[t - 1])) return mg_fail(ctx, MG_ERR_ARG, "mg_set_species: T_grid must increase");
    cudaSetDevice(ctx->device);
    drop_state(ctx);
    ctx->h_ovl_off.clear();
    ctx->n_lev = n_lev;
    ctx->n_lines = n_lines;
    ctx->n_T = n_T;
    ctx->mass = mass;
    ctx->h_E.assign(E, E + n_lev);
    ctx->h_g.assign(g, g + n_lev);
    ctx->h_Tgrid.assign(T_grid, T_grid + n_T);
    int npairs = n_lev * (n_lev - 1) / 2;
    ctx->h_Kdown.assign(K_down, K_down + (size_t)npairs * n_T);
    ctx->h_lines.resize(n_lines);
    for (int l = 0; l < n_lines; l++) {
        LineConst &c = ctx->h_lines[l];
        c.up = up[l];
        c.lo = lo[l];
        c.A = A[l];
        c.nu = (E[up[l]] - E[lo[l]]) / kH;
        c.Bul = A[l] * kC * kC / (2.0 * kH * c.nu * c.nu * c.nu);
        c.Blu = g[up[l]] / g[lo[l]] * c.Bul;
        c.pre = kH * c.nu / (4.0 * kPi);
    }
    std::vector<float> lconst(2 * n_lines);
    for (int l = 0; l < n_lines; l++) {
        lconst[l] = (float)(kC / (ctx->h_lines[l].nu * kSqrtPi) / kChiScale);
        lconst[n_lines + l] = (float)(ctx->h_lines[l].nu * 1e-9);
    }
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_lconst, 2 * n_lines))) return rc;
    if ((rc = upload(ctx, ctx->d_lconst, lconst.data(), 4 * 2 * n_lines))) return rc;
    if ((rc = mg_alloc(ctx, &ctx->d_lines, n_lines)) || (rc = mg_alloc(ctx, &ctx->d_E, n_lev)) ||
        (rc = mg_alloc(ctx, &ctx->d_g, n_lev)) || (rc = mg_alloc(ctx, &ctx->d_Tgrid, n_T)) ||
        (rc = mg_alloc(ctx, &ctx->d_Kdown, (size_t)npairs * n_T)))
        return rc;
    if ((rc = upload(ctx, ctx->d_lines, ctx->h_lines.data(), sizeof(LineConst) * n_lines)) ||
        (rc = upload(ctx, ctx->d_E, E, 8 * n_lev)) || (rc = upload(ctx, ctx->d_g, g, 8 * n_lev)) ||
        (rc = upload(ctx, ctx->d_Tgrid, T_grid, 8 * n_T)) ||
        (rc = upload(ctx, ctx->d_Kdown, K_down, 8 * (size_t)npairs * n_T)))
        return rc;
    ctx->have_species = true;
    ctx->have_pops = false;
    ctx->have_rad = false;
    ctx->coll_ready = false;
    free_rays(ctx);
    if ((rc = refresh_widths(ctx))) return rc;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    mg_noalloc_prepare(ctx);   // records its own failure; the update reports it
    return MG_OK;
}

// ------------------------------------------------------------------ directions
// HEALPix RING-scheme pixel centres (Gorski et al. 2005), walked ring by ring: polar
// rings i = 1..nside-1 hold 4i pixels at z = +-(1 - i^2/(3 nside^2)) with
// phi = (j - 1/2) pi/(2i); belt rings i = nside..3 nside hold 4 nside pixels at
// z = 4/3 - 2i/(3 nside) with phi = (j - s/2) pi/(2 nside), s = (i - nside + 1) mod 2.
static std::vector<double> healpix_ring(int nside) {
    std::vector<double> d;
    auto push = [&](double z, double phi) {
        double st = std::sqrt(std::max(0.0, (1.0 - z) * (1.0 + z)));
        d.push_back(st * std::cos(phi));
        d.push_back(st * std::sin(phi));
        d.push_back(z);
    };
    const double n2 = (double)nside * nside;
    for (int i = 1; i < nside; i++)
        for (int j = 1; j <= 4 * i; j++) push(1.0 - (double)i * i / (3.0 * n2), kPi / (2.0 * i) * (j - 0.5));
    for (int i = nside; i <= 3 * nside; i++) {
        int s = (i - nside + 1) % 2;
        for (int j = 1; j <= 4 * nside; j++)
            push(4.0 / 3.0 - 2.0 * i / (3.0 * nside), kPi / (2.0 * nside) * (j - 0.5 * s));
    }
    for (int i = nside - 1; i >= 1; i--)
        for (int j = 1; j <= 4 * i; j++) push(-(1.0 - (double)i * i / (3.0 * n2)), kPi / (2.0 * i) * (j - 0.5));
    return d;
}

static int set_dirs(mg_ctx *ctx, int R, const std::vector<double> &d) {
    std::vector<int32_t> anti(R, -1);
    for (int r = 0; r < R; r++) {
        double best = 1e300;
        for (int k = 0; k < R; k++) {
            double e = std::fabs(d[3 * k] + d[3 * r]) + std::fabs(d[3 * k + 1] + d[3 * r + 1]) +
                       std::fabs(d[3 * k + 2] + d[3 * r + 2]);
            if (e < best) { best = e; anti[r] = k; }
        }
        if (best > 1e-12) return mg_fail(ctx, MG_ERR_ARG, "directions: a direction has no antipode");
        double nn = d[3 * r] * d[3 * r] + d[3 * r + 1] * d[3 * r + 1] + d[3 * r + 2] * d[3 * r + 2];
        if (std::fabs(nn - 1.0) > 1e-12) return mg_fail(ctx, MG_ERR_ARG, "directions: not unit vectors");
    }
    ctx->R = R;
    ctx->h_dirs = d;
    ctx->h_anti = anti;
    ctx->h_pf.clear();
    ctx->h_pb.clear();
    for (int r = 0; r < R; r++)
        if (r < anti[r]) { ctx->h_pf.push_back(r); ctx->h_pb.push_back(anti[r]); }
    ctx->P = (int32_t)ctx->h_pf.size();
    if (2 * ctx->P != R) return mg_fail(ctx, MG_ERR_ARG, "directions: antipodes do not pair up");
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_dirs, 3 * R)) || (rc = mg_alloc(ctx, &ctx->d_pf, ctx->P)) ||
        (rc = mg_alloc(ctx, &ctx->d_pb, ctx->P)))
        return rc;
    if ((rc = upload(ctx, ctx->d_dirs, d.data(), 24 * R)) || (rc = upload(ctx, ctx->d_pf, ctx->h_pf.data(), 4 * ctx->P)) ||
        (rc = upload(ctx, ctx->d_pb, ctx->h_pb.data(), 4 * ctx->P)))
        return rc;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    free_rays(ctx);
    ctx->have_dirs = true;
    return MG_OK;
}

extern "C" int mg_set_directions(mg_ctx *ctx, int32_t nside) {
    if (!ctx) return MG_ERR_ARG;
    if (nside < 1 || nside > 64) return mg_fail(ctx, MG_ERR_ARG, "mg_set_directions: nside in [1, 64]");
    cudaSetDevice(ctx->device);
    return set_dirs(ctx, 12 * nside * nside, healpix_ring(nside));
}

extern "C" int mg_set_directions_custom(mg_ctx *ctx, int32_t R, const double *dirs) {
    if (!ctx) return MG_ERR_ARG;
    if (R < 2 || R % 2 || !dirs) return mg_fail(ctx, MG_ERR_ARG, "mg_set_directions_custom: need an even R >= 2");
    cudaSetDevice(ctx->device);
    return set_dirs(ctx, R, std::vector<double>(dirs, dirs + 3 * R));
}

extern "C" int mg_get_directions(const mg_ctx *ctx, int32_t *R, double *dirs, int32_t *antipode) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_dirs) return mg_fail(ctx, MG_ERR_STATE, "no directions set");
    if (R) *R = ctx->R;
    if (dirs) std::memcpy(dirs, ctx->h_dirs.data(), 24 * ctx->R);
    if (antipode) std::memcpy(antipode, ctx->h_anti.data(), 4 * ctx->R);
    return MG_OK;
}

// ------------------------------------------------------------------ quadrature
// Gauss-Hermite rule for the normalised weight exp(-x^2)/sqrt(pi): the nodes are the
// eigenvalues of the Jacobi matrix (zero diagonal, off-diagonal sqrt(k/2)), found by
// Sturm-sequence bisection; each weight is the Christoffel number
// 1 / sum_k p_k(x)^2 over the orthonormal Hermite polynomials p_0..p_{n-1}.
static int sturm_below(int n, double x) {
    // number of eigenvalues of the Jacobi matrix smaller than x
    int cnt = 0;
    double q = -x;   // d_0 - x with d = 0
    if (q < 0) cnt++;
    for (int k = 1; k < n; k++) {
        double b2 = 0.5 * k;
        if (q == 0.0) q = 1e-300;
        q = -x - b2 / q;
        if (q < 0) cnt++;
    }
    return cnt;
}

static void gauss_hermite_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    double bound = std::sqrt(2.0 * n + 1.0) + 1.0;
    for (int i = 0; i < n; i++) {
        double lo = -bound, hi = bound;   // smallest x with count > i
        for (int it = 0; it < 200 && hi - lo > 0.0; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_below(n, mid) > i) hi = mid;
            else lo = mid;
        }
        double xi = 0.5 * (lo + hi);
        // one Newton step on p_n through the recurrence
        for (int it = 0; it < 2; it++) {
            double p0 = 1.0, p1 = std::sqrt(2.0) * xi, d0 = 0.0, d1 = std::sqrt(2.0);
            if (n == 1) { p1 = p0 * std::sqrt(2.0) * xi; }
            for (int k = 1; k < n; k++) {
                double a = std::sqrt((k + 1) / 2.0), b = std::sqrt(k / 2.0);
                double p2 = (xi * p1 - b * p0) / a;
                double d2 = (p1 + xi * d1 - b * d0) / a;
                p0 = p1; p1 = p2; d0 = d1; d1 = d2;
            }
            if (d1 != 0.0 && std::isfinite(p1 / d1)) xi -= p1 / d1;
        }
        x[i] = xi;
        double s = 1.0, pm = 1.0, pc = std::sqrt(2.0) * xi;
        if (n > 1) s += pc * pc;
        for (int k = 1; k + 1 < n; k++) {
            double pn = (xi * pc - std::sqrt(k / 2.0) * pm) / std::sqrt((k + 1) / 2.0);
            s += pn * pn;
            pm = pc; pc = pn;
        }
        w[i] = 1.0 / s;
    }
}

extern "C" int mg_set_quadrature(mg_ctx *ctx, int32_t n_q) {
    if (!ctx) return MG_ERR_ARG;
    if (n_q < 1 || n_q > 128) return mg_fail(ctx, MG_ERR_ARG, "mg_set_quadrature: n_q in [1, 128]");
    cudaSetDevice(ctx->device);
    gauss_hermite_rule(n_q, ctx->h_roots, ctx->h_weights);
    ctx->Q = n_q;
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_roots, n_q)) || (rc = mg_alloc(ctx, &ctx->d_weights, n_q))) return rc;
    if ((rc = upload(ctx, ctx->d_roots, ctx->h_roots.data(), 8 * n_q)) ||
        (rc = upload(ctx, ctx->d_weights, ctx->h_weights.data(), 8 * n_q)))
        return rc;
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->have_quad = true;
    ctx->have_rad = false;
    return MG_OK;
}

extern "C" int mg_get_quadrature(const mg_ctx *ctx, double *roots, double *weights) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_quad) return mg_fail(ctx, MG_ERR_STATE, "no quadrature set");
    if (roots) std::memcpy(roots, ctx->h_roots.data(), 8 * ctx->Q);
    if (weights) std::memcpy(weights, ctx->h_weights.data(), 8 * ctx->Q);
    return MG_OK;
}

// ------------------------------------------------------------------ ray tracing
extern "C" int mg_trace_rays(mg_ctx *ctx, mg_ray_stats *out) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_mesh || !ctx->have_model || !ctx->have_species || !ctx->have_dirs)
        return mg_fail(ctx, MG_ERR_STATE, "mg_trace_rays: needs mesh, model, species and directions");
    cudaSetDevice(ctx->device);
    int rc = mg_launch_trace(ctx);
    if (rc < 0) return rc;
    if (out) {
        out->n_rays = ctx->n * ctx->R;
        out->n_elements = ctx->n_elements;
        out->n_expanded = ctx->n_expanded;
        out->max_pair_len = ctx->max_pair_len;
        out->n_dead_end = ctx->n_dead;
        out->mean_pair_len = ctx->P ? (double)(ctx->n_expanded + (int64_t)ctx->n * ctx->P) / ((double)ctx->n * ctx->P) : 0.0;
    }
    return ctx->n_dead ? MG_WARN_DEAD_END_RAYS : MG_OK;
}

extern "C" int mg_get_ray(const mg_ctx *cctx, int64_t point, int32_t ray, int32_t *cells, int32_t *nsub,
                          double *ds, double *vpar, int64_t cap, int64_t *len) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->traced) return mg_fail(ctx, MG_ERR_STATE, "mg_get_ray: rays not traced");
    if (point < 0 || point >= ctx->n || ray < 0 || ray >= ctx->R || !len)
        return mg_fail(ctx, MG_ERR_ARG, "mg_get_ray: bad point or ray");
    cudaSetDevice(ctx->device);
    int64_t off[2];
    int64_t idx = point * ctx->R + ray;
    MG_CUDA(cudaMemcpyAsync(off, ctx->d_ray_off + idx, 16, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t n = off[1] - off[0];
    *len = n;
    if (n > cap) return mg_fail(ctx, MG_ERR_ARG, "mg_get_ray: buffer too small");
    if (n == 0) return MG_OK;
    std::vector<int32_t> xc(n);
    if (cells) MG_CUDA(cudaMemcpyAsync(cells, ctx->d_cells + off[0], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(xc.data(), ctx->d_xcum + off[0], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (ds) MG_CUDA(cudaMemcpyAsync(ds, ctx->d_ds + off[0], 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (vpar) MG_CUDA(cudaMemcpyAsync(vpar, ctx->d_vpar + off[0], 8 * n, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (nsub)
        for (int64_t e = 0; e < n; e++) nsub[e] = xc[e] - (e ? xc[e - 1] : 0) - 1;
    return MG_OK;
}

// ------------------------------------------------------------------ populations
// New populations start a new iteration: the bandwidth in use returns to the option's.
void mg_band_restart(mg_ctx *ctx) {
    ctx->band_cur = ctx->opt.alo_band;
    ctx->band_gmres_iters = 0;
}

static int ensure_state(mg_ctx *ctx) {
    int64_t n = ctx->n;
    int L = ctx->n_lines, lev = ctx->n_lev;
    int rc;
    if (!ctx->d_pops) {
        if ((rc = mg_alloc(ctx, &ctx->d_pops, n * lev)) || (rc = mg_alloc(ctx, &ctx->d_pops_new, n * lev)) ||
            (rc = mg_alloc(ctx, &ctx->d_line, n * L * 2)) || (rc = mg_alloc(ctx, &ctx->d_linef, n * L * 2)) ||
            (rc = mg_alloc(ctx, &ctx->d_J, n * L)) || (rc = mg_alloc(ctx, &ctx->d_L, n * L)) ||
            (rc = mg_alloc(ctx, &ctx->d_Jeff, n * L)) || (rc = mg_alloc(ctx, &ctx->d_Lc, n * L)))
            return rc;
    }
    if (ctx->opt.spectrum && !ctx->d_Jnu && ctx->have_quad)
        if ((rc = mg_alloc(ctx, &ctx->d_Jnu, n * L * ctx->Q))) return rc;
    return MG_OK;
}

static int need_species_model(mg_ctx *ctx, const char *who) {
    if (!ctx->have_mesh || !ctx->have_model || !ctx->have_species)
        return mg_fail(ctx, MG_ERR_STATE, std::string(who) + ": needs mesh, model and species");
    return MG_OK;
}



extern "C" int mg_init_populations(mg_ctx *ctx, int32_t mode) {
    if (!ctx) return MG_ERR_ARG;
    int rc;
    if ((rc = need_species_model(ctx, "mg_init_populations"))) return rc;
    cudaSetDevice(ctx->device);
    if (mode == MG_INIT_GIVEN) {
        if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "mg_init_populations: no populations given");
        return MG_OK;
    }
    if (mode == MG_INIT_MLP) {
        if (!ctx->mlp) return mg_fail(ctx, MG_ERR_STATE, "mg_init_populations: no network attached");
        return mg_init_populations_mlp(ctx, ctx->mlp);
    }
    if (mode != MG_INIT_LTE) return mg_fail(ctx, MG_ERR_ARG, "mg_init_populations: unknown mode");
    if ((rc = ensure_state(ctx))) return rc;
    if ((rc = mg_launch_lte(ctx))) return rc;
    mg_band_restart(ctx);
    ctx->have_pops = true;
    ctx->have_rad = false;
    return MG_OK;
}

extern "C" int mg_set_populations(mg_ctx *ctx, const double *pops) {
    if (!ctx || !pops) return ctx ? mg_fail(ctx, MG_ERR_ARG, "null populations") : MG_ERR_ARG;
    int rc;
    if ((rc = need_species_model(ctx, "mg_set_populations"))) return rc;
    cudaSetDevice(ctx->device);
    if ((rc = ensure_state(ctx))) return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->d_pops, pops, 8 * ctx->n * ctx->n_lev, cudaMemcpyHostToDevice, ctx->stream));
    mg_band_restart(ctx);
    ctx->have_pops = true;
    ctx->have_rad = false;
    return MG_OK;
}

extern "C" int mg_set_populations_dev(mg_ctx *ctx, const double *d_pops) {
    if (!ctx || !d_pops) return ctx ? mg_fail(ctx, MG_ERR_ARG, "null populations") : MG_ERR_ARG;
    int rc;
    if ((rc = need_species_model(ctx, "mg_set_populations_dev"))) return rc;
    cudaSetDevice(ctx->device);
    if ((rc = ensure_state(ctx))) return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->d_pops, d_pops, 8 * ctx->n * ctx->n_lev, cudaMemcpyDeviceToDevice, ctx->stream));
    mg_band_restart(ctx);
    ctx->have_pops = true;
    ctx->have_rad = false;
    return MG_OK;
}

extern "C" int mg_get_populations(const mg_ctx *cctx, double *pops) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !pops) return MG_ERR_ARG;
    if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "no populations");
    cudaSetDevice(ctx->device);
    MG_CUDA(cudaMemcpyAsync(pops, ctx->d_pops, 8 * ctx->n * ctx->n_lev, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

extern "C" int mg_get_populations_dev(const mg_ctx *cctx, double *d_pops) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !d_pops) return MG_ERR_ARG;
    if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "no populations");
    cudaSetDevice(ctx->device);
    MG_CUDA(cudaMemcpyAsync(d_pops, ctx->d_pops, 8 * ctx->n * ctx->n_lev, cudaMemcpyDeviceToDevice, ctx->stream));
    return MG_OK;
}

// ------------------------------------------------------------------ formal solve
static int check_solve_ready(mg_ctx *ctx) {
    if (!ctx->traced) return mg_fail(ctx, MG_ERR_STATE, "formal solve: trace the rays first");
    if (!ctx->have_quad) return mg_fail(ctx, MG_ERR_STATE, "formal solve: set the quadrature first");
    if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "formal solve: set or initialise populations first");
    return MG_OK;
}

extern "C" int mg_formal_solve(mg_ctx *ctx) {
    if (!ctx) return MG_ERR_ARG;
    int rc;
    if ((rc = check_solve_ready(ctx))) return rc;
    cudaSetDevice(ctx->device);
    if ((rc = ensure_state(ctx))) return rc;
    if (ctx->h_ovl_off.size() != (size_t)ctx->n_lines + 1)
        if ((rc = upload_overlaps(ctx))) return rc;
    MG_CUDA(cudaMemsetAsync(ctx->d_scal + 4, 0, sizeof(unsigned long long), ctx->stream));
    if (ctx->band_cur > 0 && (rc = mg_band_alloc(ctx))) return rc;
    if ((rc = mg_launch_line_data(ctx))) return rc;
    if (ctx->sca_on) {
        // scattering (Sec. 3.3): the right-hand side from the previous iteration's mean
        // intensity, until the per-bin mean intensity changes by less than sca_tol
        const int64_t m = ctx->n * ctx->n_lines * ctx->Q;
        double ch = INFINITY;
        int it = 0;
        while (it < ctx->sca_max_iter) {
            if ((rc = mg_launch_feautrier(ctx))) return rc;
            if ((rc = mg_launch_max_rel_change(ctx, m, ctx->d_Jsca_new, ctx->d_Jsca, ctx->d_scaw))) return rc;
            std::swap(ctx->d_Jsca, ctx->d_Jsca_new);
            it++;
            unsigned long long bits = 0;
            MG_CUDA(cudaMemcpyAsync(&bits, ctx->d_scaw, 8, cudaMemcpyDeviceToHost, ctx->stream));
            MG_CUDA(cudaStreamSynchronize(ctx->stream));
            std::memcpy(&ch, &bits, 8);
            if (ch < ctx->sca_tol) break;
        }
        ctx->sca_iters = it;
        ctx->sca_change = ch;
        if (ctx->opt.spectrum && ctx->d_Jnu)
            MG_CUDA(cudaMemcpyAsync(ctx->d_Jnu, ctx->d_Jsca, 8 * (size_t)m, cudaMemcpyDeviceToDevice, ctx->stream));
    } else if ((rc = mg_launch_feautrier(ctx))) {
        return rc;
    }
    ctx->band_solved = ctx->opt.precision == MG_FP64 ? ctx->band_cur : 0;
    ctx->have_rad = true;
    return MG_OK;
}

extern "C" int mg_set_scattering(mg_ctx *ctx, const double *chi_sca, double tol, int32_t max_iter) {
    if (!ctx) return MG_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!chi_sca) {
        ctx->sca_on = false;
        ctx->have_rad = false;
        return MG_OK;
    }
    if (ctx->opt.precision != MG_FP64)
        return mg_fail(ctx, MG_ERR_STATE, "mg_set_scattering: scattering is built for FP64 contexts");
    if (!ctx->have_mesh || !ctx->have_species || !ctx->have_quad)
        return mg_fail(ctx, MG_ERR_STATE, "mg_set_scattering: set the mesh, species and quadrature first");
    if (!(tol > 0) || max_iter < 1) return mg_fail(ctx, MG_ERR_ARG, "mg_set_scattering: tol > 0 and max_iter >= 1");
    for (int64_t i = 0; i < ctx->n; i++)
        if (!(chi_sca[i] >= 0.0) || !std::isfinite(chi_sca[i]))
            return mg_fail(ctx, MG_ERR_ARG, "mg_set_scattering: chi_sca must be finite and >= 0");
    const size_t m = (size_t)ctx->n * ctx->n_lines * ctx->Q;
    int rc;
    if ((rc = mg_alloc(ctx, &ctx->d_chisca, ctx->n)) || (rc = mg_alloc(ctx, &ctx->d_Jsca, m)) ||
        (rc = mg_alloc(ctx, &ctx->d_Jsca_new, m)) || (rc = mg_alloc(ctx, &ctx->d_scaw, 1)))
        return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->d_chisca, chi_sca, 8 * (size_t)ctx->n, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemsetAsync(ctx->d_Jsca, 0, 8 * m, ctx->stream));   // no scattered light to start from
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->sca_tol = tol;
    ctx->sca_max_iter = max_iter;
    ctx->sca_iters = 0;
    ctx->sca_change = 0.0;
    ctx->sca_on = true;
    ctx->have_rad = false;
    return MG_OK;
}

extern "C" int mg_scattering_status(const mg_ctx *ctx, int32_t *iterations, double *last_change) {
    if (!ctx) return MG_ERR_ARG;
    if (iterations) *iterations = ctx->sca_iters;
    if (last_change) *last_change = ctx->sca_change;
    return MG_OK;
}

extern "C" int mg_get_radiation(const mg_ctx *cctx, double *J, double *L, double *Jeff) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_rad) return mg_fail(ctx, MG_ERR_STATE, "no radiation field computed");
    cudaSetDevice(ctx->device);
    size_t b = 8 * ctx->n * ctx->n_lines;
    if (J) MG_CUDA(cudaMemcpyAsync(J, ctx->d_J, b, cudaMemcpyDeviceToHost, ctx->stream));
    if (L) MG_CUDA(cudaMemcpyAsync(L, ctx->d_L, b, cudaMemcpyDeviceToHost, ctx->stream));
    if (Jeff) MG_CUDA(cudaMemcpyAsync(Jeff, ctx->d_Jeff, b, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

extern "C" int mg_set_radiation(mg_ctx *ctx, const double *J, const double *L, const double *Jeff) {
    if (!ctx) return MG_ERR_ARG;
    if (!J || !L || !Jeff) return mg_fail(ctx, MG_ERR_ARG, "mg_set_radiation: null buffer");
    int rc;
    if ((rc = need_species_model(ctx, "mg_set_radiation"))) return rc;
    if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "mg_set_radiation: set or initialise populations first");
    const size_t m = (size_t)ctx->n * ctx->n_lines;
    for (size_t i = 0; i < m; i++)
        if (!std::isfinite(J[i]) || !std::isfinite(L[i]) || !std::isfinite(Jeff[i]))
            return mg_fail(ctx, MG_ERR_ARG, "mg_set_radiation: non-finite value");
    cudaSetDevice(ctx->device);
    if ((rc = ensure_state(ctx))) return rc;
    std::vector<double> oml(m);
    for (size_t i = 0; i < m; i++) oml[i] = 1.0 - L[i];
    MG_CUDA(cudaMemcpyAsync(ctx->d_J, J, 8 * m, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(ctx->d_L, L, 8 * m, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(ctx->d_Jeff, Jeff, 8 * m, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(ctx->d_Lc, oml.data(), 8 * m, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemsetAsync(ctx->d_scal + 4, 0, sizeof(unsigned long long), ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->band_solved = 0;   // no band terms: the next update uses the diagonal ALO
    ctx->have_rad = true;
    return MG_OK;
}

extern "C" int mg_get_radiation_dev(const mg_ctx *cctx, double *J, double *L, double *Jeff) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_rad) return mg_fail(ctx, MG_ERR_STATE, "no radiation field computed");
    cudaSetDevice(ctx->device);
    size_t b = 8 * ctx->n * ctx->n_lines;
    if (J) MG_CUDA(cudaMemcpyAsync(J, ctx->d_J, b, cudaMemcpyDeviceToDevice, ctx->stream));
    if (L) MG_CUDA(cudaMemcpyAsync(L, ctx->d_L, b, cudaMemcpyDeviceToDevice, ctx->stream));
    if (Jeff) MG_CUDA(cudaMemcpyAsync(Jeff, ctx->d_Jeff, b, cudaMemcpyDeviceToDevice, ctx->stream));
    return MG_OK;
}

extern "C" int mg_get_spectrum(const mg_ctx *cctx, double *Jnu) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !Jnu) return MG_ERR_ARG;
    if (!ctx->opt.spectrum || !ctx->d_Jnu) return mg_fail(ctx, MG_ERR_STATE, "spectrum not enabled (opt.spectrum)");
    if (!ctx->have_rad) return mg_fail(ctx, MG_ERR_STATE, "no radiation field computed");
    cudaSetDevice(ctx->device);
    MG_CUDA(cudaMemcpyAsync(Jnu, ctx->d_Jnu, 8 * ctx->n * ctx->n_lines * ctx->Q, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

// ------------------------------------------------------------------ images
static int image_common(mg_ctx *ctx, int32_t ray, int32_t line, int32_t n_ch, const double *u_ch, bool dev,
                        double *I, double *xy) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->traced) return mg_fail(ctx, MG_ERR_STATE, "mg_image: trace the rays first");
    if (!ctx->have_pops) return mg_fail(ctx, MG_ERR_STATE, "mg_image: set or initialise populations first");
    if (ray < 0 || ray >= ctx->R || line < 0 || line >= ctx->n_lines || n_ch < 1 || n_ch > MG_IMAGE_MAX_CHANNELS ||
        !u_ch || !I)
        return mg_fail(ctx, MG_ERR_ARG, "mg_image: bad ray, line, channel count or null pointer");
    double umax = 0.0;
    for (int c = 0; c < n_ch; c++) {
        if (!(std::fabs(u_ch[c]) < 0.1 * kC)) return mg_fail(ctx, MG_ERR_ARG, "mg_image: channel offsets must be finite and below c/10");
        umax = std::max(umax, std::fabs(u_ch[c]));
    }
    cudaSetDevice(ctx->device);
    int rc;
    if ((rc = ensure_state(ctx))) return rc;
    // Lines within reach of the channels: for line l2, |x| >= (|dnl| - rat (umax + V (1 + umax/c)))/b_max
    // with V the largest speed, so beyond 28 widths exp(-x^2) underflows to zero and the line is left out.
    const double nu_l = ctx->h_lines[line].nu;
    std::vector<Overlap> ov;
    for (int l2 = 0; l2 < ctx->n_lines; l2++) {
        const double nu2 = ctx->h_lines[l2].nu;
        Overlap d{};
        d.dnl = kC * (nu_l - nu2) / nu2;
        d.rat = nu_l / nu2;
        d.inv_nu2 = 1.0 / nu2;
        d.l2 = l2;
        const double reach = d.rat * (umax + ctx->vmax * (1.0 + umax / kC));
        if (l2 == line || std::fabs(d.dnl) - reach <= 28.0 * ctx->bmax) ov.push_back(d);
    }
    const int64_t need = ctx->n * (int64_t)n_ch;
    if (!dev && need > ctx->img_cap) {
        if ((rc = mg_alloc(ctx, &ctx->d_img, need))) return rc;
        ctx->img_cap = need;
    }
    if (n_ch > ctx->uch_cap) {
        if ((rc = mg_alloc(ctx, &ctx->d_uch, n_ch))) return rc;
        ctx->uch_cap = n_ch;
    }
    if (!ctx->d_imgov && (rc = mg_alloc(ctx, &ctx->d_imgov, ctx->n_lines))) return rc;
    if (!ctx->d_imgxy && (rc = mg_alloc(ctx, &ctx->d_imgxy, 2 * ctx->n))) return rc;
    if (!ctx->d_imglf && (rc = mg_alloc(ctx, &ctx->d_imglf, 2 * ctx->n * ctx->n_lines))) return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->d_uch, u_ch, 8 * (size_t)n_ch, cudaMemcpyHostToDevice, ctx->stream));
    MG_CUDA(cudaMemcpyAsync(ctx->d_imgov, ov.data(), sizeof(Overlap) * ov.size(), cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = mg_launch_line_data64(ctx, ctx->d_imglf, ctx->d_scal + 6))) return rc;
    double *d_I = dev ? I : ctx->d_img;
    double *d_xy = dev ? xy : ctx->d_imgxy;
    if (!d_xy) d_xy = ctx->d_imgxy;
    if ((rc = mg_launch_image(ctx, ray, line, n_ch, ctx->d_uch, ctx->d_imgov, (int)ov.size(), d_I, d_xy))) return rc;
    if (!dev) {
        MG_CUDA(cudaMemcpyAsync(I, d_I, 8 * (size_t)need, cudaMemcpyDeviceToHost, ctx->stream));
        if (xy) MG_CUDA(cudaMemcpyAsync(xy, d_xy, 16 * (size_t)ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    int32_t err = 0;
    MG_CUDA(cudaMemcpyAsync(&err, ctx->d_err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (err) return mg_fail(ctx, MG_ERR_CAPACITY, "mg_image: a ray pair is longer than the traced maximum");
    return MG_OK;
}

extern "C" int mg_image(mg_ctx *ctx, int32_t ray, int32_t line, int32_t n_ch, const double *u_ch, double *I,
                        double *xy) {
    return image_common(ctx, ray, line, n_ch, u_ch, false, I, xy);
}

extern "C" int mg_image_dev(mg_ctx *ctx, int32_t ray, int32_t line, int32_t n_ch, const double *u_ch, double *d_I,
                            double *d_xy) {
    return image_common(ctx, ray, line, n_ch, u_ch, true, d_I, d_xy);
}

// ------------------------------------------------------------------ statistical equilibrium
extern "C" int mg_update_populations(mg_ctx *ctx, double *max_rel_change) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->have_rad) return mg_fail(ctx, MG_ERR_STATE, "mg_update_populations: run the formal solve first");
    cudaSetDevice(ctx->device);
    int rc;
    if (!ctx->coll_ready) {
        if ((rc = mg_launch_collision_rates(ctx))) return rc;
        ctx->coll_ready = true;
    }
    if (ctx->band_cur > 0 && ctx->band_solved > 0) {
        // band ALO: one coupled system over all cells, with bandwidth reduction
        if ((rc = mg_band_geometry(ctx))) return rc;
        double ch = 0.0;
        int64_t nf = 0;
        int bu = 0;
        {
            MgTimed t(ctx, "band_solve");   // block set-up, GMRES and finish, host steps included
            if ((rc = mg_band_update(ctx, &ch, &nf, &bu)) < 0) return rc;
        }
        MG_CUDA(cudaMemcpyAsync(ctx->h_scal + 4, ctx->d_scal + 4, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                ctx->stream));
        MG_CUDA(cudaStreamSynchronize(ctx->stream));
        if (max_rel_change) *max_rel_change = ch;
        ctx->have_rad = false;
        ctx->last_fallback = nf;
        ctx->last_neg_opacity = (int64_t)ctx->h_scal[4];
        if (nf) return MG_WARN_NEG_POP_FALLBACK;
        return ctx->h_scal[4] ? MG_WARN_NEG_OPACITY : MG_OK;
    }
    if ((rc = mg_launch_stateq(ctx))) return rc;
    MG_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->d_scal, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    double ch;
    std::memcpy(&ch, &ctx->h_scal[0], 8);
    if (max_rel_change) *max_rel_change = ch;
    ctx->have_rad = false;
    ctx->last_fallback = (int64_t)ctx->h_scal[1];
    ctx->last_neg_opacity = (int64_t)ctx->h_scal[4];
    if (ctx->h_scal[2]) return mg_fail(ctx, MG_ERR_NUMERIC, "statistical equilibrium: non-finite populations after fallback");
    if (ctx->h_scal[1]) return MG_WARN_NEG_POP_FALLBACK;
    return ctx->h_scal[4] ? MG_WARN_NEG_OPACITY : MG_OK;
}

extern "C" int mg_promoted_cells(const mg_ctx *cctx, int64_t *count) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !count) return MG_ERR_ARG;
    *count = 0;
    if (!ctx->d_promo) return MG_OK;
    int32_t c = 0;
    MG_CUDA(cudaMemcpyAsync(&c, ctx->d_promo + ctx->n, 4, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    *count = c;
    return MG_OK;
}

extern "C" int mg_band_status(const mg_ctx *ctx, int32_t *band_in_use, int64_t *gmres_iters) {
    if (!ctx) return MG_ERR_ARG;
    if (band_in_use) *band_in_use = ctx->band_cur;
    if (gmres_iters) *gmres_iters = ctx->band_gmres_iters;
    return MG_OK;
}

extern "C" int mg_get_band_terms(const mg_ctx *cctx, int32_t *band, double *Jeffb, double *M) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !band) return MG_ERR_ARG;
    if (!ctx->have_rad || ctx->band_solved < 1)
        return mg_fail(ctx, MG_ERR_STATE, "mg_get_band_terms: the last formal solve had no band terms");
    cudaSetDevice(ctx->device);
    const int B = ctx->band_solved;
    *band = B;
    const size_t nl = (size_t)ctx->n * ctx->n_lines;
    if (Jeffb) MG_CUDA(cudaMemcpyAsync(Jeffb, ctx->d_Jeffb, 8 * nl * B, cudaMemcpyDeviceToHost, ctx->stream));
    if (M) MG_CUDA(cudaMemcpyAsync(M, ctx->d_Mb, 8 * nl * ctx->R * B, cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

extern "C" int mg_status_counts(const mg_ctx *ctx, int64_t *fallback_cells, int64_t *negative_opacity) {
    if (!ctx) return MG_ERR_ARG;
    if (fallback_cells) *fallback_cells = ctx->last_fallback;
    if (negative_opacity) *negative_opacity = ctx->last_neg_opacity;
    return MG_OK;
}

// ------------------------------------------------------------------ ALI driver
extern "C" int mg_iterate(mg_ctx *ctx, mg_ali_report *rep) {
    if (!ctx) return MG_ERR_ARG;
    int rc;
    if ((rc = check_solve_ready(ctx))) return rc;
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();
    mg_ali_report r{};
    int nh = 0, grow = 0;
    double last = 0.0;
    for (int it = 0; it < ctx->opt.max_iter; it++) {
        if ((rc = mg_formal_solve(ctx)) < 0) return rc;
        double ch = 0;
        rc = mg_update_populations(ctx, &ch);
        if (rc < 0) return rc;
        r.n_fallback += ctx->last_fallback;
        r.iterations = it + 1;
        r.last_change = ch;
        // band ALO: a change that has grown three iterations in a row (a diverging
        // iteration) reduces the bandwidth in use by one
        grow = (it > 0 && ch > last) ? grow + 1 : 0;
        last = ch;
        if (grow >= 3 && ctx->band_cur > 0) {
            ctx->band_cur--;
            grow = 0;
        }
        if (ch < ctx->opt.tol) { r.converged = 1; break; }
        if (ctx->opt.ng_period > 0) {
            if ((rc = mg_launch_push_history(ctx))) return rc;
            if (nh < 4) nh++;
            if (nh == 4 && (it + 1) % ctx->opt.ng_period == 0) {
                int acc = 0;
                if ((rc = mg_launch_ng(ctx, &acc))) return rc;
                r.ng_steps += acc;
                nh = 0;
            }
        }
    }
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    r.alo_band = ctx->band_cur;
    if (rep) *rep = r;
    return r.converged ? MG_OK : mg_fail(ctx, MG_ERR_NOT_CONVERGED, "ALI did not reach the tolerance");
}

int mg_ensure_solve_state(mg_ctx *ctx) {
    int rc;
    if ((rc = check_solve_ready(ctx))) return rc;
    if ((rc = ensure_state(ctx))) return rc;
    if (ctx->h_ovl_off.size() != (size_t)ctx->n_lines + 1)
        if ((rc = upload_overlaps(ctx))) return rc;
    if (!ctx->coll_ready) {
        if ((rc = mg_launch_collision_rates(ctx))) return rc;
        ctx->coll_ready = true;
    }
    return MG_OK;
}

// ------------------------------------------------------------------ autotuning
extern "C" int mg_autotune(mg_ctx *ctx, int32_t reps, int32_t *variant, double *ms, int32_t *n_tried) {
    if (!ctx) return MG_ERR_ARG;
    int rc;
    if ((rc = check_solve_ready(ctx))) return rc;
    if (ctx->opt.precision != MG_MIXED) return mg_fail(ctx, MG_ERR_STATE, "mg_autotune: only the mixed path has variants");
    cudaSetDevice(ctx->device);
    if ((rc = ensure_state(ctx))) return rc;
    if (ctx->h_ovl_off.size() != (size_t)ctx->n_lines + 1)
        if ((rc = upload_overlaps(ctx))) return rc;
    if ((rc = mg_launch_line_data(ctx))) return rc;
    int b = -1, nt = 0;
    double bms = 0;
    if ((rc = mg_autotune_mixed(ctx, reps < 1 ? 1 : reps, &b, &bms, &nt))) return rc;
    if (variant) *variant = b;
    if (ms) *ms = bms;
    if (n_tried) *n_tried = nt;
    ctx->have_rad = true;
    return MG_OK;
}

extern "C" int mg_set_variant(mg_ctx *ctx, int32_t variant) {
    if (!ctx) return MG_ERR_ARG;
    ctx->mixed_variant = variant;
    return MG_OK;
}

// ------------------------------------------------------------------ timing and counts
extern "C" int mg_kernel_times(const mg_ctx *ctx, int32_t cap, const char **names, double *ms,
                               int64_t *launches, int32_t *count) {
    if (!ctx) return MG_ERR_ARG;
    int k = (int)std::min<size_t>(cap, ctx->timers.size());
    for (int i = 0; i < k; i++) {
        if (names) names[i] = ctx->timers[i].name.c_str();
        if (ms) ms[i] = ctx->timers[i].ms;
        if (launches) launches[i] = ctx->timers[i].launches;
    }
    if (count) *count = (int32_t)ctx->timers.size();
    return MG_OK;
}

extern "C" int mg_reset_kernel_times(mg_ctx *ctx) {
    if (!ctx) return MG_ERR_ARG;
    for (auto &t : ctx->timers) { t.ms = 0.0; t.launches = 0; }
    cudaSetDevice(ctx->device);
    MG_CUDA(cudaMemsetAsync(ctx->d_scal + 7, 0, sizeof(unsigned long long), ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    return MG_OK;
}

extern "C" int mg_executed_work(const mg_ctx *cctx, int64_t *updates) {
    mg_ctx *ctx = const_cast<mg_ctx *>(cctx);
    if (!ctx || !updates) return MG_ERR_ARG;
    cudaSetDevice(ctx->device);
    unsigned long long v = 0;
    MG_CUDA(cudaMemcpyAsync(&v, ctx->d_scal + 7, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    MG_CUDA(cudaStreamSynchronize(ctx->stream));
    *updates = (int64_t)v;
    return MG_OK;
}

extern "C" int mg_work_counts(const mg_ctx *ctx, int64_t *solves, int64_t *updates) {
    if (!ctx) return MG_ERR_ARG;
    if (!ctx->traced || !ctx->have_quad) return mg_fail(ctx, MG_ERR_STATE, "trace rays and set the quadrature first");
    int64_t F = (int64_t)ctx->n_lines * ctx->Q;
    if (solves) *solves = ctx->n * ctx->P * F;
    if (updates) *updates = (ctx->n_expanded + ctx->n * ctx->P) * F;
    return MG_OK;
}
