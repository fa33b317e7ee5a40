// Internal declarations shared by the translation units of libmagritte_gb300.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/magritte_gb300.h"

namespace mg {

// CODATA 2018 constants.
constexpr double kH = 6.62607015e-34;
constexpr double kKB = 1.380649e-23;
constexpr double kC = 299792458.0;
constexpr double kSqrtPi = 1.7724538509055160273;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxLev = 64;

// Scales of the FP32 formal solve: intensities in units of kI0 (W m^-2 Hz^-1 sr^-1);
// float line data hold chi_int * kChiScale and eta_int * kEtaScale = chi scale / kI0.
constexpr float kI0 = 1e-20f;
constexpr double kChiScale = 1e5;
constexpr double kEtaScale = 1e25;

// Per-line constants of the species, copied to the device once.
struct LineConst {
    double nu;      // line-centre frequency (E_u - E_l)/h
    double A;       // Einstein A_ul
    double Bul;     // A c^2 / (2 h nu^3)
    double Blu;     // (g_u/g_l) B_ul
    double pre;     // h nu / (4 pi)
    int32_t up, lo;
};

// Overlap descriptor of a (line l, other line l') pair used by the profile sum:
// x_l' = (dnl + rat * (a_q (1 - v/c) - v)) / b with dnl = c (nu_l - nu_l')/nu_l'
// and rat = nu_l/nu_l'.
struct Overlap {
    double dnl;
    double rat;
    double inv_nu2;   // 1/nu_l' (profile normalisation delta_nu = nu_l' b / c)
    int32_t l2;
    int32_t pad;
};

struct KernelTimer {
    std::string name;
    double ms = 0.0;
    int64_t launches = 0;
};

}  // namespace mg

struct mg_ctx {
    mg_options opt{};
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    mutable std::string err;

    // ---- mesh
    bool have_mesh = false;
    int64_t n = 0;
    int32_t geometry = MG_GEOM_3D;
    int64_t n_edges = 0;
    double extent = 0.0;   // longest path through the model (m): bounding-box diagonal, or the sphere's diameter
    double *d_pos = nullptr, *d_vel = nullptr;
    int64_t *d_nbr_off = nullptr;
    int32_t *d_nbr_idx = nullptr;
    uint8_t *d_bdy = nullptr;
    std::vector<double> h_T, h_vturb;      // kept to compute widths once the mass is known
    double vmax = 0.0;                     // largest |v| over the points (image line lists)
    double bmax = 0.0;                     // largest velocity width

    // ---- model
    bool have_model = false;
    double *d_ncoll = nullptr, *d_T = nullptr, *d_nspec = nullptr;
    double *d_b = nullptr;        // velocity width per point
    float *d_bf = nullptr;

    // ---- species
    bool have_species = false;
    int32_t n_lev = 0, n_lines = 0, n_T = 0;
    double mass = 0.0;
    std::vector<double> h_E, h_g, h_Tgrid, h_Kdown;
    std::vector<mg::LineConst> h_lines;
    mg::LineConst *d_lines = nullptr;
    float *d_lconst = nullptr;    // [2L]: c/(nu_l sqrt(pi))/kChiScale, nu_l in GHz (FP32 solve)
    double *d_E = nullptr, *d_g = nullptr, *d_Tgrid = nullptr, *d_Kdown = nullptr;
    double *d_coll = nullptr;     // [n][n_pairs][2] (down, up) collision rates
    bool coll_ready = false;
    std::vector<int32_t> h_ovl_off;
    std::vector<mg::Overlap> h_ovl;
    int32_t *d_ovl_off = nullptr;
    mg::Overlap *d_ovl = nullptr;

    // ---- directions
    bool have_dirs = false;
    int32_t R = 0, P = 0;
    std::vector<double> h_dirs;
    std::vector<int32_t> h_anti, h_pf, h_pb;
    double *d_dirs = nullptr;
    int32_t *d_pf = nullptr, *d_pb = nullptr;

    // ---- quadrature
    bool have_quad = false;
    int32_t Q = 0;
    std::vector<double> h_roots, h_weights;
    double *d_roots = nullptr, *d_weights = nullptr;

    // ---- ray store: per (point, ray) half-ray, CSR by point then ray
    bool traced = false;
    int64_t *d_ray_off = nullptr;  // [n*R + 1]
    int32_t *d_cells = nullptr;    // traced cell
    int32_t *d_xcum = nullptr;     // expanded points up to and including the element
    double *d_ds = nullptr;        // path length from the previous point
    double *d_vpar = nullptr;      // line-of-sight velocity relative to the origin
    float *d_dsf = nullptr, *d_vparf = nullptr;
    int64_t n_elements = 0, n_expanded = 0, max_pair_len = 0, n_dead = 0;
    int64_t work_solves = 0, work_updates = 0;

    // ---- state
    bool have_pops = false;
    double *d_pops = nullptr, *d_pops_new = nullptr;
    double *d_hist[4] = {nullptr, nullptr, nullptr, nullptr};
    double *d_ng_tmp = nullptr, *d_ng_part = nullptr;
    double *d_line = nullptr;      // [n][L][2] (eta_int, chi_int)
    float *d_linef = nullptr;
    double *d_J = nullptr, *d_L = nullptr, *d_Jeff = nullptr, *d_Lc = nullptr;
    double *d_Jnu = nullptr;
    bool have_rad = false;

    // ---- scalars
    unsigned long long *d_scal = nullptr;   // [0] max change bits, [1] fallbacks, [2] non-finite,
                                            // [3] Ng flags, [4] negative line opacities, [5] band
                                            // solve: singular blocks, [6] image negative opacities,
                                            // [7] executed point-bin updates (profiling)
    int64_t last_fallback = 0, last_neg_opacity = 0;
    unsigned long long *h_scal = nullptr;   // pinned
    int32_t *d_err = nullptr;               // kernel error word

    // ---- FP64 promotion of optically thick cells (mixed precision)
    mg_mlp *mlp = nullptr;        // attached network for MG_INIT_MLP (not owned)
    int32_t *d_promo = nullptr;   // [n] origin list, then [n] count in d_promo[n]

    // ---- images: channel offsets, candidate lines, output buffers (grow-only)
    double *d_uch = nullptr, *d_img = nullptr, *d_imgxy = nullptr;
    mg::Overlap *d_imgov = nullptr;
    float *d_imglf = nullptr;      // [n][L][2] FP32 (eta_int, chi_int) for the FP32 image kernel
    int64_t img_cap = 0;
    int32_t uch_cap = 0;

    // ---- launch variant of the mixed formal solve (-1: default for the model)
    int mixed_variant = -1;

    // ---- band-diagonal ALO (band.cu): bandwidth in use, that of the last formal solve,
    //      its J_eff of bandwidths 1..B [B][n][L] and coupling terms [n][L][R][B], the
    //      band points' cells and weights [n][R][opt.alo_band], and the solver's buffers
    int band_cur = 0, band_solved = 0;
    bool band_geo_ready = false;
    int64_t band_cap_n = 0;
    int band_cap_lev = 0, band_cap_L = 0, band_cap_R = 0;
    int64_t band_gmres_iters = 0;
    double *d_Jeffb = nullptr, *d_Mb = nullptr;
    int2 *d_bcells = nullptr;
    double *d_bw = nullptr, *d_blu = nullptr, *d_bs = nullptr, *d_bz = nullptr, *d_bx = nullptr, *d_bw2 = nullptr;
    double *d_bV = nullptr, *d_bpart = nullptr, *d_bh = nullptr;
    int32_t *d_bpiv = nullptr;

    // ---- isotropic coherent scattering (FP64): opacity [n], the previous and the new mean
    //      intensity per bin [n][L][Q], the iteration's tolerance, cap and last outcome
    bool sca_on = false;
    double *d_chisca = nullptr, *d_Jsca = nullptr, *d_Jsca_new = nullptr;
    unsigned long long *d_scaw = nullptr;
    double sca_tol = 1e-8, sca_change = 0.0;
    int32_t sca_max_iter = 100, sca_iters = 0;

    // ---- allocation-free update: set-up done at mg_set_species (stateq_noalloc.cu)
    bool na_ready = false;
    std::string na_error;
    unsigned long long *na_scratch = nullptr;   // device address of the static scratch

    // ---- profiling
    std::vector<mg::KernelTimer> timers;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// ---------------------------------------------------------------- helpers
int mg_fail(const mg_ctx *ctx, int code, const std::string &msg);
int mg_cuda_check(const mg_ctx *ctx, cudaError_t e, const char *what);
#define MG_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return mg_cuda_check(ctx, e_, #call);      \
    } while (0)

template <typename T>
int mg_alloc(mg_ctx *ctx, T **p, size_t count) {
    if (*p) { cudaFree(*p); *p = nullptr; }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return mg_fail(ctx, MG_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    return MG_OK;
}
template <typename T>
void mg_free(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Kernel timing scope: records events around a launch when opt.profile is set.
struct MgTimed {
    mg_ctx *ctx;
    int idx;
    MgTimed(mg_ctx *c, const char *name);
    ~MgTimed();
};

// ---------------------------------------------------------------- launchers
int mg_launch_trace(mg_ctx *ctx);
int mg_launch_line_data(mg_ctx *ctx);
int mg_launch_line_data_mixed(mg_ctx *ctx);
int mg_launch_line_data64(mg_ctx *ctx, float *linef, unsigned long long *neg);
int mg_launch_image(mg_ctx *ctx, int ray, int line, int n_ch, const double *d_u, const mg::Overlap *d_ov,
                    int n_ov, double *d_I, double *d_xy);
int mg_launch_feautrier(mg_ctx *ctx);
int mg_launch_max_rel_change(mg_ctx *ctx, int64_t m, const double *a_new, const double *a_old,
                             unsigned long long *word);
int mg_launch_feautrier_fp64_list(mg_ctx *ctx, const int32_t *olist, const int32_t *ocount);
int mg_autotune_mixed(mg_ctx *ctx, int reps, int *best, double *best_ms, int *n_tried);
int mg_launch_lte(mg_ctx *ctx);
int mg_launch_collision_rates(mg_ctx *ctx);
int mg_launch_stateq(mg_ctx *ctx);
int mg_launch_ng(mg_ctx *ctx, int *accepted);
int mg_launch_push_history(mg_ctx *ctx);
int mg_launch_stateq_into(mg_ctx *ctx, const double *pops_old, double *pops_new, const int32_t *active);
int mg_ensure_solve_state(mg_ctx *ctx);   // state buffers, overlaps and collision rates ready
void mg_noalloc_prepare(mg_ctx *ctx);     // set-up of mg_update_populations_noalloc
int mg_band_alloc(mg_ctx *ctx);
int mg_band_geometry(mg_ctx *ctx);
int mg_band_update(mg_ctx *ctx, double *max_change, int64_t *n_fallback, int *band_used);
void mg_band_free(mg_ctx *ctx);
void mg_band_restart(mg_ctx *ctx);        // populations set: bandwidth back to opt.alo_band
// batch helpers (solve_mixed.cu)
size_t mg_mixargs_size();
int mg_fill_mixargs(mg_ctx *ctx, void *out);
int mg_variant_count();
int mg_variant_valid(int v, int L, int Q);
int mg_variant_minb(int v);
int mg_variant_g(int v);
int mg_variant_default(int L, int Q);
int mg_variant_effective(const mg_ctx *ctx, int v);
int mg_batch_launch(int v, int grid, const void *d_args, const void *d_items, int64_t n_items,
                    unsigned long long *counter, const int32_t *active, cudaStream_t stream);
