/*
 * magritte_gb300.h -- C ABI of the GB300 (sm_103a) implementation of the accelerated
 * Lambda iteration (ALI) hot path of non-LTE line radiative transfer described in
 * De Ceuster et al. 2019, "Magritte I" (arXiv:1912.08445).
 *
 * Steps behind this boundary, each in hand-written CUDA kernels:
 *   ray tracing by neighbour walk (Sec. 3.2), Gauss-Hermite frequency bins (Sec. 3.1.2),
 *   HEALPix directions (Sec. 3.1.3), Doppler-shifted Gaussian line profiles (Sec. 2.2.1),
 *   the second-order Feautrier solve of each ray pair with the diagonal approximate
 *   Lambda operator (Sec. 3.3, 3.4, eq. 'GFE', 'ALO', 'ourJeff'), per-cell statistical
 *   equilibrium (eq. 'ourALI'), the validity check (Sec. 6.1), Ng acceleration
 *   (Sec. 3.4), and images from the outward radiation on each point's ray pair (Sec. 3.5).
 *
 * Conventions
 *   - Units are SI: m, m/s, K, m^-3, J, s^-1, m^3 s^-1. Intensities are W m^-2 Hz^-1 sr^-1.
 *   - Every function returns an int status: MG_OK (0), a negative error code, or a
 *     positive warning. mg_last_error() gives a message for the last non-OK status.
 *   - Ownership: the caller owns every host array it passes. Setters copy the data in;
 *     the library keeps no caller pointer. Getters copy into caller buffers of the
 *     documented size. The context owns all device memory it allocates.
 *   - Functions ending in _dev take device pointers (on the context's device) and read
 *     or write them in stream order on the context's stream; they never free them.
 *   - A context is not thread safe; distinct contexts are independent.
 *   - A call on a context makes the context's device the calling thread's current CUDA
 *     device and leaves it so (mg_measure_pipe_rates restores the previous one).
 *   - Array layouts are C order (row major); "[n][3]" means 3 doubles per point.
 */
#ifndef MAGRITTE_GB300_H
#define MAGRITTE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MG_OK                      0
#define MG_ERR_ARG               (-1)  /* invalid argument, size or layout              */
#define MG_ERR_STATE             (-2)  /* call out of order (e.g. solve before tracing) */
#define MG_ERR_CUDA              (-3)  /* a CUDA runtime call failed                    */
#define MG_ERR_OOM               (-4)  /* device or host allocation failed              */
#define MG_ERR_NOT_CONVERGED     (-5)  /* ALI reached max_iter above tolerance          */
#define MG_ERR_NUMERIC           (-6)  /* non-finite result that no fallback repaired   */
#define MG_ERR_CAPACITY          (-7)  /* a ray pair exceeds the kernel's staging limit */
#define MG_WARN_DEAD_END_RAYS      1   /* some rays ended at a cell with no farther neighbour */
#define MG_WARN_NEG_POP_FALLBACK   2   /* some cells fell back to plain Lambda iteration    */
#define MG_WARN_NEG_OPACITY        3   /* some line opacity integral was negative (population
                                          inversion, a maser): the opacity floor was applied  */

/* precision of the formal solve */
#define MG_FP64   0   /* everything in FP64                                              */
#define MG_MIXED  1   /* formal solve in FP32; statistical equilibrium in FP64           */

/* geometry of a mesh */
#define MG_GEOM_3D            0  /* point cloud with neighbour lists                     */
#define MG_GEOM_SPHERICAL_1D  1  /* spherically symmetric shells: points on the +z axis at
                                    increasing radii; radii below the first form an empty
                                    core (a first radius of 0 is a centre point)          */

/* initial populations */
#define MG_INIT_LTE    0
#define MG_INIT_GIVEN  1   /* keep what mg_set_populations stored */
#define MG_INIT_MLP    2   /* the network attached with mg_attach_mlp (see below) */

typedef struct mg_ctx mg_ctx;

typedef struct {
    int32_t precision;     /* MG_FP64 or MG_MIXED                                         */
    int32_t device;        /* CUDA device ordinal                                         */
    double  tol;           /* ALI stops when the max relative population change < tol     */
    int32_t max_iter;      /* ALI iteration cap                                           */
    int32_t ng_period;     /* Ng step every ng_period iterations from 4 iterates; 0 = off */
    double  dshift_frac;   /* velocity-step limit as a fraction of the local line width  */
    double  chi_min;       /* opacity floor, m^-1                                         */
    double  dtau_min;      /* optical-depth increment floor                               */
    double  T_cmb;         /* temperature of the incoming boundary black body, K          */
    double  line_cut;      /* lines farther than line_cut widths from a bin are skipped   */
    int64_t max_steps;     /* cap on traced cells per half-ray                            */
    int32_t profile;       /* 1: time each kernel launch with CUDA events                 */
    int32_t spectrum;      /* 1: keep the per-bin mean intensity for mg_get_spectrum      */
    int32_t pad;
    double  tau_fp64;      /* MG_MIXED only: cells whose largest diagonal ALO weight L is
                              >= 1 - 1/tau_fp64 (optically thick lines) are solved again in
                              FP64 after the FP32 pass; 0 = off                            */
    int32_t alo_band;      /* MG_FP64 only: bandwidth b of the approximate Lambda operator
                              (Sec. 3.4, eq. 'ALO'): the entries |k - ko| <= b of the
                              inverse's row along every ray pair; 0 = diagonal, at most 2   */
    int32_t pad2;
} mg_options;

/* Fills *opt with defaults: MG_FP64, device 0, tol 1e-6, max_iter 300, ng_period 4,
 * dshift_frac 1/3, chi_min 1e-30, dtau_min 1e-30, T_cmb 2.725, line_cut 7.5,
 * max_steps 100000, profile 0, spectrum 0, tau_fp64 0 (off), alo_band 0 (diagonal). */
void mg_default_options(mg_options *opt);

/* Creates a context on opt->device (NULL opt = defaults). *out receives the handle.
 * Errors: MG_ERR_ARG (bad option), MG_ERR_CUDA (device unusable). */
int mg_create(mg_ctx **out, const mg_options *opt);
int mg_destroy(mg_ctx *ctx);
const char *mg_last_error(const mg_ctx *ctx);

/* Uses the given cudaStream_t (as void*) for all later work, e.g. a PyTorch stream; NULL
 * restores the context's own stream. The caller keeps the stream alive. */
int mg_set_stream(mg_ctx *ctx, void *stream);

/* Spatial discretisation (Sec. 3.1.1): n points, positions pos[n][3] and velocities
 * vel[n][3], neighbour lists in CSR form (nbr_off[n+1] int64, nbr_idx[nbr_off[n]] int32,
 * indices in [0, n)), boundary flags is_bdy[n] (1 = on the convex hull). For
 * MG_GEOM_SPHERICAL_1D the points lie on +z with increasing radius and vel is radial
 * (along z). Errors: MG_ERR_ARG on bad sizes or indices. Invalidates traced rays. */
int mg_set_mesh(mg_ctx *ctx, int64_t n, const double *pos, const double *vel,
                const int64_t *nbr_off, const int32_t *nbr_idx, const uint8_t *is_bdy,
                int32_t geometry);

/* Per-point physical fields [n]: collision-partner density, temperature, turbulent
 * velocity and species density (Sec. 2.2.1). Requires mg_set_mesh first. */
int mg_set_model(mg_ctx *ctx, const double *n_coll, const double *T, const double *v_turb,
                 const double *n_species);

/* Species (Sec. 2.2.1): n_lev levels with energies E (J) and weights g, mass (kg);
 * n_lines radiative lines up[l] -> lo[l] (up > lo in energy) with Einstein A (s^-1);
 * collisional de-excitation coefficients K_down[(n_lev(n_lev-1)/2)][n_T] (m^3 s^-1) on
 * the temperature grid T_grid[n_T], pairs ordered (1,0),(2,0),(2,1),(3,0),...
 * Einstein B follow from A; excitation coefficients follow by detailed balance,
 * C_lu = C_ul (g_u/g_l) exp(-(E_u - E_l)/kT). Limits: n_lev <= 64. */
int mg_set_species(mg_ctx *ctx, int32_t n_lev, const double *E, const double *g, double mass,
                   int32_t n_lines, const int32_t *up, const int32_t *lo, const double *A,
                   int32_t n_T, const double *T_grid, const double *K_down);

/* Ray directions: HEALPix pixel centres for nside (12 nside^2 rays, Sec. 3.1.3), or R
 * custom unit vectors dirs[R][3]. Every direction must have an exact antipode in the
 * set (ray pairs, Sec. 3.3). Invalidates traced rays. */
int mg_set_directions(mg_ctx *ctx, int32_t nside);
int mg_set_directions_custom(mg_ctx *ctx, int32_t R, const double *dirs);
/* Copies the directions [R][3] and antipode indices [R] into caller buffers. */
int mg_get_directions(const mg_ctx *ctx, int32_t *R, double *dirs, int32_t *antipode);

/* Gauss-Hermite frequency bins per line (Sec. 3.1.2): n_q roots r_q and the
 * profile-normalised weights (sum 1). Limits: 1 <= n_q <= 128. */
int mg_set_quadrature(mg_ctx *ctx, int32_t n_q);
int mg_get_quadrature(const mg_ctx *ctx, double *roots, double *weights);

typedef struct {
    int64_t n_rays;          /* n * R half-rays                                    */
    int64_t n_elements;      /* traced cells over all half-rays                    */
    int64_t n_expanded;      /* cells plus points inserted by the velocity-step rule */
    int64_t max_pair_len;    /* longest ray pair in expanded points, origin included */
    int64_t n_dead_end;      /* half-rays that ended at a cell with no farther neighbour */
    double  mean_pair_len;   /* mean expanded ray-pair length                      */
} mg_ray_stats;

/* Traces every (point, direction) half-ray on the device (Sec. 3.2): from the current
 * cell, step to the neighbour with a strictly larger projection on the ray that lies
 * closest to the ray (ties: smaller squared distance, then smaller projection, then
 * smaller index); stop after a boundary cell or at a dead end. Between consecutive
 * points, ceil(dv/(f min(b_a, b_b))) - 1 points are inserted when the line-of-sight
 * velocity step dv exceeds f = dshift_frac of the smaller local width. Requires mesh,
 * model and directions. Returns MG_WARN_DEAD_END_RAYS when some rays dead-ended. */
int mg_trace_rays(mg_ctx *ctx, mg_ray_stats *out);

/* Copies half-ray (point, ray): cells[len] (traced cell indices), nsub[len] (points
 * inserted before each cell), ds[len] (path length from the previous point, m) and
 * vpar[len] (line-of-sight velocity relative to the origin, m/s). cap is the buffer
 * length; *len receives the ray length (MG_ERR_ARG if it exceeds cap). */
int mg_get_ray(const mg_ctx *ctx, int64_t point, int32_t ray, int32_t *cells, int32_t *nsub,
               double *ds, double *vpar, int64_t cap, int64_t *len);

/* Level populations [n][n_lev] (m^-3). mg_init_populations(MG_INIT_LTE) sets Boltzmann
 * populations at the local temperature. */
int mg_init_populations(mg_ctx *ctx, int32_t mode);
int mg_set_populations(mg_ctx *ctx, const double *pops);
int mg_get_populations(const mg_ctx *ctx, double *pops);
int mg_set_populations_dev(mg_ctx *ctx, const double *d_pops);
int mg_get_populations_dev(const mg_ctx *ctx, double *d_pops);

/* Formal solution from the current populations (Sec. 3.3-3.4): for every point, ray
 * pair and frequency bin, solves the Feautrier equation along the pair and forms, per
 * point and line,
 *   J    = (1/P) sum_pairs sum_q w_q u,                       (mean intensity)
 *   L    = (1/P) sum sum w_q Lambda*_oo chi_l/chi,            (diagonal ALO weight)
 *   Jeff = (1/P) sum sum w_q (u - Lambda*_oo eta_l/chi).      (effective intensity)
 * Requires traced rays, quadrature, species and populations. Asynchronous. */
int mg_formal_solve(mg_ctx *ctx);
/* Copies J, L, Jeff, each [n][n_lines], to host buffers (any may be NULL). */
int mg_get_radiation(const mg_ctx *ctx, double *J, double *L, double *Jeff);
int mg_get_radiation_dev(const mg_ctx *ctx, double *d_J, double *d_L, double *d_Jeff);
/* Replaces the radiation field that mg_update_populations reads: J, L and Jeff, each
 * [n][n_lines] host buffers (all three required), stand for the result of a formal solve
 * (eq. 'L_operator', 'ourJeff'), e.g. a field computed elsewhere or one saved with
 * mg_get_radiation; 1 - L is formed from L. Requires populations (MG_ERR_STATE);
 * MG_ERR_ARG for a null buffer or a non-finite value. Clears the negative-opacity count
 * of the last formal solve. Synchronises. */
int mg_set_radiation(mg_ctx *ctx, const double *J, const double *L, const double *Jeff);
/* Per-bin mean intensity (1/P) sum_pairs u, [n][n_lines][n_q]; needs opt.spectrum = 1. */
int mg_get_spectrum(const mg_ctx *ctx, double *Jnu);

/* Isotropic, coherent scattering (Sec. 2.1 eq. 'RTE', Sec. 3.3 eq. 'RTE2', 'GFE'), FP64
 * contexts: chi_sca [n] (m^-1, >= 0) is a frequency-independent scattering opacity per
 * point that scatters isotropically and keeps the comoving frequency. Then chi+ = chi_sca,
 * chi- = 0, Psi- = 0 and Psi+ = chi_sca J_nu, and eq. 'GFE' for u is the second-order
 * equation with opacity chi + chi_sca and source (eta + chi_sca J)/(chi + chi_sca). As
 * Sec. 3.3 prescribes, its right-hand side is evaluated with the previous iteration's
 * solution: every mg_formal_solve repeats the formal solution, with J per point and bin
 * from the previous pass (read at a ray point's comoving offset from the line centre,
 * in units of the point's width, from the bins of line l of the point's cells, linear
 * between the Gauss-Hermite roots, interpolated between the cells like the line data),
 * until the per-bin mean intensity changes by less than tol relative, or max_iter passes.
 * The first pass of the first solve starts from no scattered light; later solves start
 * from the last one's field. J, L, J_eff and the spectrum are those of the last pass
 * (L and J_eff with the total opacity in their denominators). NULL chi_sca switches
 * scattering off. Images leave the scattered light out. MG_ERR_STATE in mixed
 * contexts or before the mesh, species and quadrature; MG_ERR_ARG for a negative or
 * non-finite value. Setting the mesh or species switches scattering off. */
int mg_set_scattering(mg_ctx *ctx, const double *chi_sca, double tol, int32_t max_iter);
/* Passes and final relative change of the scattering iteration of the last formal solve. */
int mg_scattering_status(const mg_ctx *ctx, int32_t *iterations, double *last_change);

/* Image of the model along ray direction `ray` (Sec. 3.5, 'Imaging the model'): every
 * point o contributes one image point, its projection on the plane orthogonal to
 * n = dirs[ray], carrying the intensity that leaves the model along n on the ray pair
 * through o.
 *   ray      in [0, R): the direction n (the pair is ray and its antipode);
 *   line     in [0, n_lines): reference line of the channels;
 *   u_ch     [n_ch] host: channel c has rest-frame frequency nu_line (1 + u_ch[c]/c)
 *            (velocity units, as the formal solve's bins r_q b_o); |u_ch| < c/10;
 *   I        [n][n_ch] output intensity, W m^-2 Hz^-1 sr^-1;
 *   xy       [n][2] output sky-plane coordinates (x.e1, x.e2), e1 = (z x n)/|z x n|
 *            (x in place of z when |n_z| >= 0.9), e2 = n x e1; NULL allowed.
 * Method: along the pair's points (those of the formal solve: traced cells, inserted
 * points, interpolated line data, floors, trapezoidal dtau) the intensity is carried
 * from the far end of the -n half, where the CMB enters at its comoving frequency, to
 * the far end of the n half with the first-order equation dI/dtau = S - I, the source
 * linear in tau between points (Olson & Kunasz 1987). At a point of velocity v the
 * comoving frequency is nu (1 - n.v/c). All lines whose profiles reach the channels add
 * to opacity and emissivity, from the current populations. An FP64 context computes
 * in FP64; a mixed-precision context in FP32 (FP64 when more than 4 lines reach the
 * channels or the FP32 staging does not fit in shared memory).
 * Requires traced rays and populations (MG_ERR_STATE otherwise); 1 <= n_ch <=
 * MG_IMAGE_MAX_CHANNELS (MG_ERR_ARG otherwise). Synchronises the context's stream. */
#define MG_IMAGE_MAX_CHANNELS 4096
int mg_image(mg_ctx *ctx, int32_t ray, int32_t line, int32_t n_ch, const double *u_ch, double *I, double *xy);
/* mg_image into device buffers d_I [n][n_ch] and d_xy [n][2] (d_xy may be NULL); u_ch
 * stays a host array. Synchronises the context's stream. */
int mg_image_dev(mg_ctx *ctx, int32_t ray, int32_t line, int32_t n_ch, const double *u_ch, double *d_I,
                 double *d_xy);

/* Statistical equilibrium with the ALO (eq. 'ourALI') for every cell, the validity check
 * (Sec. 6.1) and the convergence measure: *max_rel_change = max over cells and levels
 * with n_i >= 1e-10 n of |n_new - n_old| / n_new (NULL allowed).
 * Diagonal ALO (bandwidth in use 0): per cell; a cell with negative or non-finite
 * populations is solved again without the ALO.
 * Band ALO (opt.alo_band > 0, bandwidth in use b > 0): the rate equations of all cells
 * form one linear system, since the upper population at the band points along every ray
 * pair (interpolated between their cells) enters the equations of the origin with the
 * coefficients of the last formal solve; it is solved by preconditioned GMRES. If a
 * population comes out negative or non-finite, or GMRES misses its tolerance, it is
 * solved again with bandwidth b - 1, down to the diagonal ALO; the bandwidth in use keeps
 * the reduction until populations are set or initialised again (mg_band_status).
 * Returns MG_WARN_NEG_POP_FALLBACK when some cell fell back, else MG_WARN_NEG_OPACITY
 * when the last formal solve met a negative line opacity integral. Synchronises. */
int mg_update_populations(mg_ctx *ctx, double *max_rel_change);

/* Allocation-free variant of mg_update_populations for callers that cannot allocate
 * device memory when they update populations (an allocator that owns the GPU's memory,
 * a loop that cannot take the synchronisation an allocation may cause, a fixed memory
 * budget). The paper has no counterpart: it is an interface addition only.
 * d_pops_old [n][n_lev] (read) and d_pops_new [n][n_lev] (written) are caller-owned
 * device buffers on the context's device; the radiation field is the one left by the
 * last mg_formal_solve or mg_set_radiation (MG_ERR_STATE otherwise). Computes the same
 * statistical equilibrium, validity fallback and convergence measure as
 * mg_update_populations, with the same return codes (MG_WARN_NEG_POP_FALLBACK, else
 * MG_WARN_NEG_OPACITY after a formal solve that met a negative opacity integral), without
 * touching the context's populations. *max_rel_change and *n_fallback (either may be
 * NULL) receive the convergence measure and the number of fallback cells.
 * It uses the diagonal ALO: MG_ERR_STATE while a band ALO is in use (opt.alo_band > 0),
 * whose coupled solve needs buffers of its own.
 * Scratch: a static 512 KiB device array per GPU that loads the library (held until
 * exit); at most 2,097,152 cells per call (MG_ERR_CAPACITY beyond). Everything that may
 * allocate -- loading the kernels and the array on the device, looking up the array's
 * device address, and reserving the kernel's local memory with a warm-up launch -- is
 * done by mg_set_species; if that set-up failed, this call returns MG_ERR_CUDA with the
 * reason. The call itself allocates nothing. It ends by synchronising the context's
 * stream, so it cannot be used inside a stream capture. Calls that overlap on the GPU
 * (other streams, threads or contexts) race on the shared scratch. */
int mg_update_populations_noalloc(mg_ctx *ctx, const double *d_pops_old, double *d_pops_new,
                                  double *max_rel_change, int64_t *n_fallback);

/* Band ALO state: *band_in_use = the bandwidth the next update starts from, *iters = GMRES
 * iterations since the populations were last set or initialised (either may be NULL). */
int mg_band_status(const mg_ctx *ctx, int32_t *band_in_use, int64_t *gmres_iters);
/* Band terms of the last FP64 formal solve with bandwidth B = *band (> 0): Jeffb
 * [B][n][n_lines] (J_eff of bandwidths 1..B, eq. 'ourJeff' with the band of the ALO) and
 * M [n][n_lines][R][B]: the coefficient with which A_ul times the upper population at the
 * j-th point from the origin of half-ray r enters the rate equation of the origin
 * (either buffer may be NULL). MG_ERR_STATE when the last formal solve had no band. */
int mg_get_band_terms(const mg_ctx *ctx, int32_t *band, double *Jeffb, double *M);

/* Counts behind the warnings of the last mg_update_populations: cells that fell back
 * without the ALO, and (point, line) pairs with a negative opacity integral in the last
 * formal solve. Either pointer may be NULL. */
int mg_status_counts(const mg_ctx *ctx, int64_t *fallback_cells, int64_t *negative_opacity);
/* Number of cells the last mixed-precision formal solve solved again in FP64
 * (opt.tau_fp64 > 0). Synchronises. */
int mg_promoted_cells(const mg_ctx *ctx, int64_t *count);

typedef struct {
    int32_t iterations;      /* regular iterations done                            */
    int32_t ng_steps;        /* Ng extrapolations accepted                         */
    int32_t converged;       /* 1 when the last change < tol                       */
    int32_t alo_band;        /* bandwidth of the ALO in use at the end             */
    double  last_change;     /* max relative change of the last iteration          */
    int64_t n_fallback;      /* cells that fell back, summed over iterations       */
    double  seconds;         /* wall time of the loop                              */
} mg_ali_report;

/* Accelerated Lambda iteration from the current populations: formal solve ->
 * statistical equilibrium -> convergence, with an Ng step every opt.ng_period
 * iterations (Sec. 3.4, 6.1), until the change < opt.tol or opt.max_iter. With a band
 * ALO, the bandwidth in use also drops by one when the change has grown in three
 * consecutive iterations (a diverging iteration).
 * Returns MG_ERR_NOT_CONVERGED when the cap is reached (populations are kept). */
int mg_iterate(mg_ctx *ctx, mg_ali_report *rep);

/* Autotuner of the mixed-precision formal solve: times every launch variant of the
 * Feautrier kernel that suits the model (lines per warp 1/2/4, bins per lane 1/2/4/8,
 * blocks per SM, warps per block, far-wing skipping on or off; 32 variants, indices 0-31,
 * those valid for the model's lines and bins tried; CUDA events, best of reps launches
 * after one warm-up) on the current populations,
 * keeps the fastest for later solves and reports it. Leaves a valid radiation field.
 * Requires precision MG_MIXED, traced rays, quadrature and populations. */
int mg_autotune(mg_ctx *ctx, int32_t reps, int32_t *variant, double *ms, int32_t *n_tried);
/* Selects a launch variant by index (-1: the model's default). Invalid indices fall back
 * to the default at launch. */
int mg_set_variant(mg_ctx *ctx, int32_t variant);

/* ---- Batches of independent models (uneven sizes) --------------------------------
 * A batch runs the ALI of many contexts together: every iteration is one CUDA graph
 * (line data of every model, one persistent formal-solve launch whose warps take work
 * items from a queue ordered by decreasing ray length, statistical equilibrium of every
 * model), and converged models drop out through device-side flags.
 * The contexts must be traced and populated, on the same device, in MG_MIXED precision,
 * with the same number of lines and bins and no overlapping lines. The batch keeps the
 * context pointers but does not own the contexts: destroy the batch first. While a batch
 * call runs, the contexts use the batch's stream. In the batch ALI each model takes its
 * own Ng steps (opt.ng_period of its context; 0 = off) between the graph launches, as in
 * mg_iterate. */
typedef struct mg_batch mg_batch;
int mg_batch_create(mg_batch **out, int32_t n_models, mg_ctx *const *models);
int mg_batch_destroy(mg_batch *batch);
const char *mg_batch_last_error(const mg_batch *batch);
/* Formal solve of every model (line data + one persistent launch). Synchronises. */
int mg_batch_formal_solve(mg_batch *batch);
/* ALI of every model to its own opt.tol / the first model's opt.max_iter; reps[n_models]
 * (may be NULL) receives per-model reports. MG_ERR_NOT_CONVERGED if some model did not
 * converge. */
int mg_batch_iterate(mg_batch *batch, mg_ali_report *reps);
/* Autotuner of the batched launch: times every valid kernel variant with the work queue
 * in cost order and in natural order (CUDA events, best of reps after a warm-up) and keeps
 * the fastest. Leaves a valid radiation field in every model. */
int mg_batch_autotune(mg_batch *batch, int32_t reps, int32_t *variant, int32_t *sorted, double *ms);
/* Sets the launch variant of the persistent kernel (an index as for mg_set_variant) and the
 * order of its work queue (sorted != 0: longest origins first; 0: natural order). A
 * variant that is not valid for the batch's (n_lines, n_q) gives MG_ERR_ARG and leaves
 * the previous choice; -1 restores the default. Invalidates the captured graph. */
int mg_batch_set_variant(mg_batch *batch, int32_t variant, int32_t sorted);
/* Sum of mg_work_counts over the batch's models. */
int mg_batch_work_counts(const mg_batch *batch, int64_t *solves, int64_t *cell_freq_updates);

/* ---- Learned initial populations (an addition to the paper's method) ---------------
 * A network maps four features of a cell -- log10 n_coll, log10 T, log10 |grad v| (the
 * least-squares velocity gradient over the neighbours) and log10 of the Sobolev optical
 * depth of line 0 at LTE -- to its log fractional level populations: 4 -> 128 -> 128 ->
 * 128 -> n_out, ReLU, log-softmax. Inference and training run in hand-written kernels:
 * BF16 tensor-core products (FP32 accumulation) for the 128-wide layers and the
 * back-propagated deltas, FP32 weight gradients, Adam on FP32 master weights. The ALI
 * from such a start converges to the same fixed point as from LTE. */
typedef struct mg_mlp mg_mlp;
typedef struct {
    int32_t epochs;      /* passes over the rows                   */
    int32_t batch;       /* rows per Adam step (>= 64)             */
    float   lr;          /* Adam learning rate                     */
    int32_t pad;
    uint64_t seed;       /* row shuffling                          */
} mg_train_opts;
typedef struct {
    double  first_loss;  /* mean loss of the first epoch           */
    double  last_loss;   /* mean loss of the last epoch            */
    int64_t steps;       /* Adam steps                             */
    double  seconds;
} mg_train_report;
/* Creates a network with n_out outputs (2 <= n_out <= 32) on a device, He-uniform weights
 * from seed. Parameters are one flat float vector: W1 [4][128], b1, W2 [128][128], b2,
 * W3, b3, W4 [128][n_out], b4 (weights stored [in][out]). */
int mg_mlp_create(mg_mlp **out, int32_t n_out, uint64_t seed, int32_t device);
int mg_mlp_destroy(mg_mlp *mlp);
const char *mg_mlp_last_error(const mg_mlp *mlp);
int mg_mlp_param_count(const mg_mlp *mlp, int64_t *count);
int mg_mlp_set_params(mg_mlp *mlp, const float *theta, int64_t count);   /* resets Adam */
int mg_mlp_get_params(const mg_mlp *mlp, float *theta, int64_t count);
/* Input normalisation f' = (f - mean)/std, mean[4], std[4] > 0. */
int mg_mlp_set_normalisation(mg_mlp *mlp, const float *mean, const float *std);
/* Host rows: X [rows][4] raw features -> logp [rows][n_out] log fractions. */
int mg_mlp_forward(mg_mlp *mlp, int64_t rows, const float *X, float *logp);
/* Loss (mean squared error of log fractions over targets Y >= 1e-12, Y [rows][n_out]
 * fractions) and its gradient [param_count] (either may be NULL). */
int mg_mlp_loss_grad(mg_mlp *mlp, int64_t rows, const float *X, const float *Y, double *loss, float *grad);
/* Adam training on host rows (copied to the device once). */
int mg_mlp_train(mg_mlp *mlp, int64_t rows, const float *X, const float *Y, const mg_train_opts *opts,
                 mg_train_report *report);
/* Features of every cell of a context, out [n][4]. */
int mg_features(mg_ctx *ctx, float *out);
/* Initial populations from the network (n_out must equal n_lev); cells whose output is
 * not finite keep LTE populations (their count: mg_status_counts' fallback_cells). */
int mg_init_populations_mlp(mg_ctx *ctx, mg_mlp *mlp);
/* Attaches a network to the context (NULL detaches) for mg_init_populations(ctx,
 * MG_INIT_MLP), which then does what mg_init_populations_mlp does. The context keeps the
 * pointer and does not own the network: the caller keeps it alive while attached.
 * MG_ERR_ARG if its outputs differ from the species' level count (when the species is set);
 * mg_init_populations(MG_INIT_MLP) without an attached network gives MG_ERR_STATE. */
int mg_attach_mlp(mg_ctx *ctx, mg_mlp *mlp);
/* Writes the network (output count, parameters and input normalisation; not the Adam
 * moments) to a file: the 8 bytes "MGMLP001", int32 n_out, int32 0, int64 n_params,
 * float mean[4], float std[4], float theta[n_params], little-endian. MG_ERR_ARG for a
 * file that cannot be written. */
int mg_mlp_save(const mg_mlp *mlp, const char *path);
/* Creates a network on `device` from a file written by mg_mlp_save. MG_ERR_ARG for a
 * missing, short or foreign file; *out is then NULL. */
int mg_mlp_load(mg_mlp **out, const char *path, int32_t device);

/* Kernel timing (opt.profile = 1): total milliseconds and launch counts per kernel
 * since the last reset, for up to cap kernels; names[i] points to static strings. */
int mg_kernel_times(const mg_ctx *ctx, int32_t cap, const char **names, double *ms,
                    int64_t *launches, int32_t *count);
int mg_reset_kernel_times(mg_ctx *ctx);

/* Algorithmic work of one formal solve: ray-pair solves (points x pairs x bins) and
 * cell-frequency updates (sum over solves of the expanded pair length). */
int mg_work_counts(const mg_ctx *ctx, int64_t *solves, int64_t *cell_freq_updates);
/* Point-bin updates the mixed-precision warp kernel executed (points swept, far-wing
 * points it skipped left out; each half-ray sweeps the origin once) since the last
 * mg_reset_kernel_times, counted only with opt.profile = 1. */
int mg_executed_work(const mg_ctx *ctx, int64_t *updates);

/* Measured throughput of the FP32 pipes that bound the mixed-precision formal solve, on
 * `device`: rates[0] scalar FFMA flops/s (2 per FMA), rates[1] packed FFMA2 flops/s,
 * rates[2] ex2.approx results/s, rates[3] rcp.approx results/s (independent chains over a
 * grid of 8 CTAs of 256 threads per SM, best of three timed launches). Allocates 16 bytes;
 * synchronises; the calling thread's current device is restored on return. */
int mg_measure_pipe_rates(int32_t device, double *rates);

#ifdef __cplusplus
}
#endif

#endif /* MAGRITTE_GB300_H */
