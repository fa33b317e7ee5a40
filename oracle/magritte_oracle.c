/*
 * FP64 CPU oracle of the accelerated-Lambda-iteration hot path of
 * De Ceuster et al., "Magritte I" (arXiv:1912.08445).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA
 * path is checked against. Only the tests, the smoke check and the bench's CPU
 * baseline may load it. It shares no code, header or table with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction, so that
 * the ray tracer's floating-point decisions are reproducible bit for bit).
 *
 * Every function follows the paper's section or equation named in its comment.
 * Readings where the paper is silent or ambiguous are marked "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Physical constants (CODATA 2018). The paper lists none; its printed line widths
 * (Sec. 4.1.1, 4.1.2) are reproduced with these values. */
static const double H_PLANCK = 6.62607015e-34;
static const double K_BOLTZ = 1.380649e-23;
static const double C_LIGHT = 299792458.0;
static const double SQRT_PI = 1.7724538509055160273;

/* Model, species, discretisation and options, all host arrays owned by the caller. */
typedef struct {
    int64_t n;
    int32_t geometry;          /* 0: 3D point cloud, 1: spherically symmetric shells on +z */
    int32_t pad0;
    const double *pos;         /* [n][3] */
    const double *vel;         /* [n][3] */
    const int64_t *nbr_off;    /* [n+1] */
    const int32_t *nbr_idx;
    const uint8_t *is_bdy;     /* [n] */
    const double *n_coll;      /* [n] collision partner density */
    const double *T;           /* [n] */
    const double *v_turb;      /* [n] */
    const double *n_spec;      /* [n] */
    int32_t n_lev;
    int32_t n_lines;
    const double *E;           /* [n_lev] */
    const double *g;           /* [n_lev] */
    double mass;
    const int32_t *up;         /* [n_lines] */
    const int32_t *lo;
    const double *A;
    int32_t n_T;
    int32_t pad1;
    const double *T_grid;      /* [n_T] */
    const double *K_down;      /* [n_lev(n_lev-1)/2][n_T] pair order (1,0),(2,0),(2,1),... */
    int32_t R;                 /* number of ray directions */
    int32_t Q;                 /* frequency bins per line */
    const double *dirs;        /* [R][3] */
    const int32_t *antipode;   /* [R] */
    const double *roots;       /* [Q] */
    const double *weights;     /* [Q] */
    double dshift_frac;        /* velocity step as a fraction of the local width */
    double chi_min;            /* opacity floor, m^-1 */
    double dtau_min;           /* optical-depth increment floor */
    double T_cmb;              /* boundary black-body temperature */
    int64_t max_steps;         /* per half-ray cap on traced cells */
} or_model;

/* ------------------------------------------------------------------ line data */

/* Line-centre frequency nu_ij = (E_i - E_j)/h. */
static double line_nu(const or_model *m, int l) {
    return (m->E[m->up[l]] - m->E[m->lo[l]]) / H_PLANCK;
}

/* Einstein B coefficients from A (textbook relations; the paper takes A from LAMDA):
 * B_ul = A_ul c^2 / (2 h nu^3), B_lu = (g_u/g_l) B_ul. */
static void einstein_b(const or_model *m, int l, double *Bul, double *Blu) {
    double nu = line_nu(m, l);
    *Bul = m->A[l] * C_LIGHT * C_LIGHT / (2.0 * H_PLANCK * nu * nu * nu);
    *Blu = m->g[m->up[l]] / m->g[m->lo[l]] * (*Bul);
}

/* Velocity width b = sqrt(v_thermal^2 + v_turb^2), v_thermal = sqrt(2 k T / m_spec)
 * (Sec. 2.2.1, characteristic line width delta_nu = nu/c * b). Operation order is
 * fixed because the ray tracer compares velocity steps against it bit for bit. */
double or_width(const or_model *m, int64_t c) {
    double vth2 = 2.0 * K_BOLTZ * m->T[c] / m->mass;
    return sqrt(vth2 + m->v_turb[c] * m->v_turb[c]);
}

/* Emissivity and opacity line integrals without the profile (eq. 'lines'):
 * eta_int = h nu/4pi n_u A_ul, chi_int = h nu/4pi (n_l B_lu - n_u B_ul). */
static void line_integrals(const or_model *m, const double *pops, int64_t c, int l,
                           double *eta_int, double *chi_int) {
    double nu = line_nu(m, l), Bul, Blu;
    einstein_b(m, l, &Bul, &Blu);
    double nu_ = pops[c * m->n_lev + m->up[l]];
    double nl_ = pops[c * m->n_lev + m->lo[l]];
    double pre = H_PLANCK * nu / (4.0 * M_PI);
    *eta_int = pre * nu_ * m->A[l];
    *chi_int = pre * (nl_ * Blu - nu_ * Bul);
}

/* Planck function B_nu(T). */
static double planck(double nu, double T) {
    return 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) / (exp(H_PLANCK * nu / (K_BOLTZ * T)) - 1.0);
}

/* LTE (Boltzmann) populations: n_i = n g_i exp(-E_i/kT) / sum_j g_j exp(-E_j/kT). */
int or_lte(const or_model *m, double *pops) {
    for (int64_t c = 0; c < m->n; c++) {
        double Z = 0.0;
        for (int i = 0; i < m->n_lev; i++) Z += m->g[i] * exp(-m->E[i] / (K_BOLTZ * m->T[c]));
        for (int i = 0; i < m->n_lev; i++)
            pops[c * m->n_lev + i] = m->n_spec[c] * m->g[i] * exp(-m->E[i] / (K_BOLTZ * m->T[c])) / Z;
    }
    return 0;
}

/* ------------------------------------------------------------------ ray tracing */

/* Half-ray from origin o along direction r (Sec. 3.2, Fig. 'ray_tracing'):
 * from the current cell, take the neighbour whose projection on the ray lies strictly
 * farther than the current cell's and which lies closest to the ray; stop after a
 * boundary cell.
 * Readings: ties go to the smaller squared distance, then the smaller projection, then
 * the smaller index; a cell with no farther neighbour ends the ray as a dead end; the
 * origin itself never stops the walk.
 * Outputs per element e (the origin is not an element): cell index, the number of
 * points inserted before it by the velocity-step rule, the path length from the
 * previous point, and the line-of-sight velocity n.(v_e - v_o). */
static int trace_3d(const or_model *m, int64_t o, int r, int64_t cap, int32_t *cells,
                    double *ds, double *vpar, int64_t *len, int *dead_end) {
    const double *n = &m->dirs[3 * r];
    const double *xo = &m->pos[3 * o];
    int64_t cur = o;
    double s_cur = 0.0;
    *len = 0;
    *dead_end = 0;
    for (;;) {
        int64_t best = -1;
        double bs = 0.0, bd2 = 0.0;
        for (int64_t e = m->nbr_off[cur]; e < m->nbr_off[cur + 1]; e++) {
            int64_t c = m->nbr_idx[e];
            double dx = m->pos[3 * c + 0] - xo[0];
            double dy = m->pos[3 * c + 1] - xo[1];
            double dz = m->pos[3 * c + 2] - xo[2];
            double s = dx * n[0] + dy * n[1] + dz * n[2];
            if (!(s > s_cur)) continue;
            double px = dx - s * n[0], py = dy - s * n[1], pz = dz - s * n[2];
            double d2 = px * px + py * py + pz * pz;
            int better = (best < 0) || (d2 < bd2) || (d2 == bd2 && s < bs) ||
                         (d2 == bd2 && s == bs && c < best);
            if (better) { best = c; bs = s; bd2 = d2; }
        }
        if (best < 0) { *dead_end = 1; break; }
        if (*len >= cap) return -1;
        const double *vb = &m->vel[3 * best], *vo = &m->vel[3 * o];
        cells[*len] = (int32_t)best;
        ds[*len] = bs - s_cur;
        vpar[*len] = n[0] * (vb[0] - vo[0]) + n[1] * (vb[1] - vo[1]) + n[2] * (vb[2] - vo[2]);
        (*len)++;
        s_cur = bs;
        cur = best;
        if (m->is_bdy[best]) break;
    }
    return 0;
}

/* Spherically symmetric model (points on the +z axis at increasing radii r_j): a ray
 * from r_o with mu = n.z crosses sphere j where s = -r_o mu +- sqrt(r_j^2 - r_o^2(1-mu^2));
 * the elements are the crossings in increasing s. Reading: radii below the innermost
 * point form an empty core; the chord across it carries no optical depth (path length 0),
 * as in the paper's power-law model with an empty core (Sec. 4.1.2). A centre point
 * (r_0 = 0) is a single point, not a sphere. */
static int trace_sph1d(const or_model *m, int64_t o, int r, int64_t cap, int32_t *cells,
                       double *ds, double *vpar, int64_t *len) {
    const double *n = &m->dirs[3 * r];
    double mu = n[2];
    double ro = m->pos[3 * o + 2];
    double p2 = ro * ro * (1.0 - mu * mu);   /* squared impact parameter */
    double vro = m->vel[3 * o + 2];
    int64_t N = m->n;
    *len = 0;
    double s_prev = 0.0;
    /* inward leg: shells o-1 .. jmin on the near side (only when mu < 0) */
    int64_t j = o;
    int through_core = 0;
    if (mu < 0.0 && ro > 0.0) {
        for (j = o - 1; j >= 0; j--) {
            double rj = m->pos[3 * j + 2];
            double q = rj * rj - p2;
            if (rj == 0.0 && p2 == 0.0) {
                /* a radial ray passes through the centre point itself */
                double s = -ro * mu;
                if (*len >= cap) return -1;
                cells[*len] = (int32_t)j;
                ds[*len] = s - s_prev;
                vpar[*len] = -vro * mu;
                (*len)++;
                s_prev = s;
                j--;
                break;
            }
            if (!(q > 0.0) || rj == 0.0) break;
            double s = -ro * mu - sqrt(q);
            if (*len >= cap) return -1;
            cells[*len] = (int32_t)j;
            ds[*len] = s - s_prev;
            vpar[*len] = m->vel[3 * j + 2] * (ro * mu + s) / rj - vro * mu;
            (*len)++;
            s_prev = s;
        }
        if (j < 0 && m->pos[2] > 0.0) through_core = 1;
        j = j + 1;   /* innermost shell crossed on the near side (or o itself) */
        if (j == 0 && m->pos[2] == 0.0) j = 1;   /* the centre point has no far side */
    }
    /* outward leg: far-side crossings of shells j .. N-1 (plus shell o when going in) */
    int64_t jstart;
    if (mu < 0.0 && ro > 0.0) jstart = j;           /* turning shell and outwards */
    else jstart = o + 1;                              /* straight out */
    for (int64_t k = jstart; k < N; k++) {
        double rk = m->pos[3 * k + 2];
        double q = rk * rk - p2;
        if (q < 0.0) continue;
        double s = -ro * mu + sqrt(q);
        if (!(s > s_prev) && !(through_core && k == jstart)) continue;
        if (*len >= cap) return -1;
        cells[*len] = (int32_t)k;
        if (through_core && k == jstart) { ds[*len] = 0.0; }
        else ds[*len] = s - s_prev;
        vpar[*len] = (rk > 0.0 ? m->vel[3 * k + 2] * (ro * mu + s) / rk : 0.0) - vro * mu;
        (*len)++;
        s_prev = s;
    }
    return 0;
}

/* Velocity-step rule (Sec. 3.1.1 and 3.2): when the line-of-sight velocity changes by
 * more than a fraction f of the local width between consecutive points, insert
 * ceil(dv/(f*min(b_a,b_b))) - 1 interpolated points. The previous point of element 0
 * is the origin (line-of-sight velocity 0). */
static void velocity_steps(const or_model *m, int64_t o, int64_t len, const int32_t *cells,
                           const double *vpar, int32_t *nsub) {
    double va = 0.0, ba = or_width(m, o);
    for (int64_t e = 0; e < len; e++) {
        double vb = vpar[e], bb = or_width(m, cells[e]);
        double dv = fabs(vb - va);
        double wmin = ba < bb ? ba : bb;
        double lim = m->dshift_frac * wmin;
        nsub[e] = 0;
        if (dv > lim) nsub[e] = (int32_t)ceil(dv / lim) - 1;
        va = vb; ba = bb;
    }
}

int or_trace(const or_model *m, int64_t o, int r, int64_t cap, int32_t *cells, int32_t *nsub,
             double *ds, double *vpar, int64_t *len, int *dead_end) {
    int rc;
    *dead_end = 0;
    if (m->geometry == 1) rc = trace_sph1d(m, o, r, cap, cells, ds, vpar, len);
    else rc = trace_3d(m, o, r, cap, cells, ds, vpar, len, dead_end);
    if (rc) return rc;
    velocity_steps(m, o, *len, cells, vpar, nsub);
    return 0;
}

/* ------------------------------------------------------------------ Feautrier solve */

/* Second-order transfer equation d^2u/dtau^2 = u - S on one ray pair (eq. 'GFE' with no
 * scattering), discretised on K points with increments dtau[0..K-2]:
 *   interior:  -A_k u_{k-1} + (1 + A_k + C_k) u_k - C_k u_{k+1} = S_k,
 *              A_k = 2/((dtau_{k-1}+dtau_k) dtau_{k-1}), C_k = 2/((dtau_{k-1}+dtau_k) dtau_k);
 *   ends (Auer 1967 second-order boundary condition with incoming intensity I):
 *              (1 + 2/dtau + 2/dtau^2) u_0 - (2/dtau^2) u_1 = S_0 + (2/dtau) I_0, mirrored.
 * Solved with the Rybicki & Hummer (1991) elimination, which carries the row excess
 * H_k = B_k - A_k - C_k separately (1 in the interior, 1 + 2/dtau at the ends):
 *   F_k = (H_k + A_k F_{k-1}/(1+F_{k-1})) / C_k,  z_k = (R_k + A_k z_{k-1}) / (C_k (1+F_k)),
 *   u_k = z_k + u_{k+1}/(1+F_k);
 * the diagonal of the inverse (the local approximate Lambda operator) follows from the
 * forward F and the backward G recursions:
 *   (T^-1)_kk = 1 / (H_k + A_k F_{k-1}/(1+F_{k-1}) + C_k G_{k+1}/(1+G_{k+1})).
 * Returns u at index ko and (T^-1)_{ko,ko}. Work arrays: 5*K doubles. */
int or_feautrier(int64_t K, int64_t ko, const double *dtau, const double *S, double I0,
                 double IK, double *u_o, double *lam_o, double *work) {
    if (K == 1) { *u_o = 0.5 * (I0 + IK); *lam_o = 0.0; return 0; }
    double *A = work, *C = work + K, *H = work + 2 * K, *F = work + 3 * K, *z = work + 4 * K;
    for (int64_t k = 0; k < K; k++) {
        if (k == 0) {
            A[k] = 0.0; C[k] = 2.0 / (dtau[0] * dtau[0]); H[k] = 1.0 + 2.0 / dtau[0];
        } else if (k == K - 1) {
            A[k] = 2.0 / (dtau[k - 1] * dtau[k - 1]); C[k] = 0.0; H[k] = 1.0 + 2.0 / dtau[k - 1];
        } else {
            A[k] = 2.0 / ((dtau[k - 1] + dtau[k]) * dtau[k - 1]);
            C[k] = 2.0 / ((dtau[k - 1] + dtau[k]) * dtau[k]);
            H[k] = 1.0;
        }
    }
    /* right-hand side */
    #define RHS(k) ((k) == 0 ? S[0] + 2.0 / dtau[0] * I0 : \
                    ((k) == K - 1 ? S[K - 1] + 2.0 / dtau[K - 2] * IK : S[k]))
    /* forward elimination */
    F[0] = H[0] / C[0];
    z[0] = RHS(0) / (H[0] + C[0]);
    for (int64_t k = 1; k < K - 1; k++) {
        F[k] = (H[k] + A[k] * F[k - 1] / (1.0 + F[k - 1])) / C[k];
        z[k] = (RHS(k) + A[k] * z[k - 1]) / (C[k] * (1.0 + F[k]));
    }
    /* last row and back substitution down to ko */
    double u = (RHS(K - 1) + A[K - 1] * z[K - 2]) / (H[K - 1] + A[K - 1] * F[K - 2] / (1.0 + F[K - 2]));
    for (int64_t k = K - 2; k >= ko; k--) u = z[k] + u / (1.0 + F[k]);
    *u_o = u;
    #undef RHS
    /* backward recursion G from the far end down to ko+1 */
    double Gn = 0.0;   /* G_{ko+1} */
    int have_G = 0;
    if (ko < K - 1) {
        double G = H[K - 1] / A[K - 1];
        for (int64_t k = K - 2; k > ko; k--) G = (H[k] + C[k] * G / (1.0 + G)) / A[k];
        Gn = G; have_G = 1;
    }
    double diag = H[ko];
    if (ko > 0) diag += A[ko] * F[ko - 1] / (1.0 + F[ko - 1]);
    if (have_G) diag += C[ko] * Gn / (1.0 + Gn);
    *lam_o = 1.0 / diag;
    return 0;
}

/* Entries (T^-1)_{ko,k}, |k - ko| <= band, of row ko of the inverse of the Feautrier
 * matrix T of or_feautrier: the weight of the source at point k in u at ko, i.e. row ko
 * of the matrix of the discretised operator (1 - D^2)^-1 of eq. 'L_operator' (Sec. 3.4),
 * whose band is the band-diagonal ALO of that section. Each entry is u at ko for a unit
 * source at point k and no incoming intensity (column k of the inverse, read at row ko),
 * from or_feautrier's elimination and back substitution. (Plain Gaussian elimination of
 * T or T^T loses every digit where an interval has a floored, near-zero optical depth:
 * the diagonal cancels against the neighbour terms there.) x[k] is written for those k
 * only. Work: 6*K doubles. Returns -1 for K < 2. */
int or_feautrier_band(int64_t K, int64_t ko, int64_t band, const double *dtau, double *x, double *work) {
    if (K < 2) return -1;
    double *e = work + 5 * K;
    for (int64_t k = 0; k < K; k++) e[k] = 0.0;
    int64_t k0 = ko - band < 0 ? 0 : ko - band, k1 = ko + band > K - 1 ? K - 1 : ko + band;
    for (int64_t k = k0; k <= k1; k++) {
        double u, lam;
        e[k] = 1.0;
        or_feautrier(K, ko, dtau, e, 0.0, 0.0, &u, &lam, work);
        e[k] = 0.0;
        x[k] = u;
    }
    return 0;
}

/* One expanded point of a ray pair: position and per-line data (interpolated for the
 * points inserted by the velocity-step rule). */
typedef struct {
    int64_t K, ko, cap;
    double *dsk;      /* [K-1] path length between points k and k+1 */
    double *vpar;     /* [K] line-of-sight velocity relative to the origin (half-ray sign) */
    double *b;        /* [K] velocity width */
    double *eta;      /* [n_lines][K] eta_int */
    double *chi;      /* [n_lines][K] chi_int */
    int64_t *ca, *cb; /* [K] cells the point interpolates between ... */
    double *w;        /* [K] ... with weight w on cb */
} pair_pts;

static int pair_alloc(pair_pts *p, int64_t cap, int nl) {
    p->cap = cap;
    p->dsk = malloc(sizeof(double) * cap);
    p->vpar = malloc(sizeof(double) * cap);
    p->b = malloc(sizeof(double) * cap);
    p->eta = malloc(sizeof(double) * cap * nl);
    p->chi = malloc(sizeof(double) * cap * nl);
    p->ca = malloc(sizeof(int64_t) * cap); p->cb = malloc(sizeof(int64_t) * cap);
    p->w = malloc(sizeof(double) * cap);
    return (p->dsk && p->vpar && p->b && p->eta && p->chi && p->ca && p->cb && p->w) ? 0 : -1;
}
static void pair_free(pair_pts *p) {
    free(p->dsk); free(p->vpar); free(p->b); free(p->eta); free(p->chi); free(p->ca); free(p->cb); free(p->w);
}

/* Per-cell line integrals for all cells (eq. 'lines' without the profile). */
static void all_line_integrals(const or_model *m, const double *pops, double *eta_c, double *chi_c) {
    for (int64_t c = 0; c < m->n; c++)
        for (int l = 0; l < m->n_lines; l++)
            line_integrals(m, pops, c, l, &eta_c[l * m->n + c], &chi_c[l * m->n + c]);
}

/* Points of one half-ray in order of increasing distance from the origin, each
 * original element preceded by its inserted points (linear interpolation with weight
 * j/(nsub+1) between the previous point and the element). Calls emit() per point. */
static int64_t expand_half(const or_model *m, int64_t o, int64_t len, const int32_t *cells,
                           const int32_t *nsub, const double *ds, const double *vpar,
                           const double *eta_c, const double *chi_c,
                           double *o_ds, double *o_v, double *o_b, double *o_eta, double *o_chi,
                           int64_t stride, int64_t cap, int64_t *o_ca, int64_t *o_cb, double *o_w) {
    int nl = m->n_lines;
    int64_t cnt = 0;
    int64_t prev = o;
    double pv = 0.0;
    for (int64_t e = 0; e < len; e++) {
        int64_t c = cells[e];
        int ns = nsub[e];
        for (int j = 1; j <= ns + 1; j++) {
            double w = (double)j / (double)(ns + 1);
            if (cnt >= cap) return -1;
            o_ds[cnt] = ds[e] / (double)(ns + 1);
            o_v[cnt] = (1.0 - w) * pv + w * vpar[e];
            o_b[cnt] = (1.0 - w) * or_width(m, prev) + w * or_width(m, c);
            if (o_ca) { o_ca[cnt] = prev; o_cb[cnt] = c; o_w[cnt] = w; }
            for (int l = 0; l < nl; l++) {
                o_eta[l * stride + cnt] = (1.0 - w) * eta_c[l * m->n + prev] + w * eta_c[l * m->n + c];
                o_chi[l * stride + cnt] = (1.0 - w) * chi_c[l * m->n + prev] + w * chi_c[l * m->n + c];
            }
            cnt++;
        }
        prev = c;
        pv = vpar[e];
    }
    return cnt;
}

/* Formal solution at a list of origin points (Sec. 3.3 and 3.4):
 * for each ray pair p and each line l and Gauss-Hermite bin q, the frequency at the
 * origin is nu = nu_l + r_q delta_nu_l(o); at every point along the pair the opacity and
 * emissivity sum the Gaussian profiles of all lines at the Doppler-shifted frequency;
 * dtau = (chi_k + chi_{k+1})/2 * ds; the pair is solved for u and the diagonal ALO.
 * Outputs per origin and line (Sec. 3.4, eq. 'L_operator', 'ALO', 'ourJeff'):
 *   J    = (1/P) sum_p sum_q w_q u,
 *   L    = (1/P) sum_p sum_q w_q Lambda*_oo chi_l/chi,
 *   Jeff = (1/P) sum_p sum_q w_q (u - Lambda*_oo eta_l/chi),
 * with P = R/2 ray pairs. Reading: the 1/2 in eq. 'L_operator' turns the average over
 * all rays into the average over ray pairs, since u(n) = u(-n).
 * The Doppler-shifted profile argument x = (nu s - nu_l')/delta_nu_l'(k), with comoving
 * factor s = 1 - v_par/c (the paper's Hubble-Lemaitre formula, eq. 'optical_depth'), is
 * evaluated in velocity units, x = (c (nu_l-nu_l')/nu_l' + (nu_l/nu_l')(r_q b_o (1 - v/c) - v)) / b_k,
 * which is the same expression without the cancellation of nu s - nu_l'.
 * Jnu (optional, [n_orig][n_lines][Q]) = (1/P) sum_p u per bin. */
/* Mean intensity of cell c in the bins of line l at offset r (in units of the width)
 * from the line centre: linear interpolation of Jnu[c][l][q] between the Gauss-Hermite
 * roots r_q (ascending), the outermost values beyond them. */
static double spectrum_at(const or_model *m, const double *Jnu, int64_t c, int l, double r) {
    const double *Jc = Jnu + ((size_t)c * m->n_lines + l) * m->Q;
    const double *x = m->roots;
    int Q = m->Q;
    if (Q == 1 || r <= x[0]) return Jc[0];
    if (r >= x[Q - 1]) return Jc[Q - 1];
    int q = 0;
    while (x[q + 1] <= r) q++;
    double t = (r - x[q]) / (x[q + 1] - x[q]);
    return Jc[q] + t * (Jc[q + 1] - Jc[q]);
}

static int formal_solve_impl(const or_model *m, const double *pops, int64_t n_orig, const int64_t *origins,
                             double *J, double *L, double *Jeff, double *Jnu, int band, double *Jeffb,
                             double *Mb, const double *chi_sca, const double *Jsca, int nthreads) {
    int nl = m->n_lines, Q = m->Q, R = m->R;
    int64_t N = m->n;
    double *eta_c = malloc(sizeof(double) * N * nl), *chi_c = malloc(sizeof(double) * N * nl);
    if (!eta_c || !chi_c) return -2;
    all_line_integrals(m, pops, eta_c, chi_c);
    int npairs = 0;
    int32_t *pf = malloc(sizeof(int32_t) * R), *pb = malloc(sizeof(int32_t) * R);
    for (int r = 0; r < R; r++) if (r < m->antipode[r]) { pf[npairs] = r; pb[npairs] = m->antipode[r]; npairs++; }
    int err = 0;
    int64_t cap = m->max_steps;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 1) reduction(|:err)
#endif
    for (int64_t io = 0; io < n_orig; io++) {
        int64_t o = origins[io];
        int32_t *cf = malloc(sizeof(int32_t) * cap), *cb = malloc(sizeof(int32_t) * cap);
        int32_t *nf = malloc(sizeof(int32_t) * cap), *nb = malloc(sizeof(int32_t) * cap);
        double *dsf = malloc(sizeof(double) * cap), *dsb = malloc(sizeof(double) * cap);
        double *vf = malloc(sizeof(double) * cap), *vb = malloc(sizeof(double) * cap);
        int64_t ecap = 0;
        double *hds = NULL, *hv = NULL, *hb = NULL, *heta = NULL, *hchi = NULL, *hw = NULL;
        int64_t *hca = NULL, *hcb = NULL;
        double *chi = NULL, *eta = NULL, *S = NULL, *dtau = NULL, *work = NULL;
        pair_pts P; P.cap = 0; P.dsk = P.vpar = P.b = P.eta = P.chi = P.w = NULL; P.ca = P.cb = NULL;
        double *accJ = calloc(nl, sizeof(double)), *accL = calloc(nl, sizeof(double)), *accE = calloc(nl, sizeof(double));
        double *accN = calloc((size_t)nl * Q, sizeof(double));
        /* band ALO: J_eff per bandwidth 1..band, coupling coefficients per (line, ray, slot) */
        double *accEb = band > 0 ? calloc((size_t)band * nl, sizeof(double)) : NULL;
        double *accM = band > 0 ? calloc((size_t)nl * R * band, sizeof(double)) : NULL;
        double *xrow = NULL, *rwork = NULL, *phil = NULL;
        if (!cf || !cb || !nf || !nb || !dsf || !dsb || !vf || !vb || !accN || (band > 0 && (!accEb || !accM))) {
            err |= 1; continue;
        }
        double bo = or_width(m, o);
        for (int p = 0; p < npairs; p++) {
            int64_t lf, lb; int de;
            if (or_trace(m, o, pf[p], cap, cf, nf, dsf, vf, &lf, &de)) { err |= 2; break; }
            if (or_trace(m, o, pb[p], cap, cb, nb, dsb, vb, &lb, &de)) { err |= 2; break; }
            int64_t need = 1;
            for (int64_t e = 0; e < lf; e++) need += nf[e] + 1;
            for (int64_t e = 0; e < lb; e++) need += nb[e] + 1;
            if (need > ecap) {
                ecap = 2 * need;
                free(hds); free(hv); free(hb); free(heta); free(hchi); pair_free(&P);
                free(chi); free(eta); free(S); free(dtau); free(work); free(hca); free(hcb); free(hw);
                hds = malloc(sizeof(double) * ecap); hv = malloc(sizeof(double) * ecap); hb = malloc(sizeof(double) * ecap);
                hca = malloc(sizeof(int64_t) * ecap); hcb = malloc(sizeof(int64_t) * ecap); hw = malloc(sizeof(double) * ecap);
                heta = malloc(sizeof(double) * ecap * nl); hchi = malloc(sizeof(double) * ecap * nl);
                chi = malloc(sizeof(double) * ecap); eta = malloc(sizeof(double) * ecap);
                S = malloc(sizeof(double) * ecap); dtau = malloc(sizeof(double) * ecap);
                work = malloc(sizeof(double) * 5 * ecap);
                free(xrow); free(rwork); free(phil);
                xrow = malloc(sizeof(double) * ecap); rwork = malloc(sizeof(double) * 6 * ecap);
                phil = malloc(sizeof(double) * ecap);
                if (pair_alloc(&P, ecap, nl) || !hds || !hv || !hb || !heta || !hchi || !chi || !eta || !S || !dtau || !work
                    || !xrow || !rwork || !phil || !hca || !hcb || !hw) { err |= 1; break; }
            }
            /* backward half expanded, then reversed into pair order */
            int64_t eb = expand_half(m, o, lb, cb, nb, dsb, vb, eta_c, chi_c, hds, hv, hb, heta, hchi, ecap, ecap,
                                     hca, hcb, hw);
            if (eb < 0) { err |= 4; break; }
            int64_t K = 0;
            for (int64_t k = eb - 1; k >= 0; k--) {
                P.vpar[K] = hv[k]; P.b[K] = hb[k];
                P.ca[K] = hca[k]; P.cb[K] = hcb[k]; P.w[K] = hw[k];
                for (int l = 0; l < nl; l++) { P.eta[l * P.cap + K] = heta[l * ecap + k]; P.chi[l * P.cap + K] = hchi[l * ecap + k]; }
                P.dsk[K] = hds[k];  /* distance from this point to the next one towards the origin */
                K++;
            }
            P.ko = K;
            P.vpar[K] = 0.0; P.b[K] = bo;
            P.ca[K] = o; P.cb[K] = o; P.w[K] = 0.0;
            for (int l = 0; l < nl; l++) { P.eta[l * P.cap + K] = eta_c[l * N + o]; P.chi[l * P.cap + K] = chi_c[l * N + o]; }
            K++;
            int64_t ef = expand_half(m, o, lf, cf, nf, dsf, vf, eta_c, chi_c, hds, hv, hb, heta, hchi, ecap, ecap,
                                     hca, hcb, hw);
            if (ef < 0) { err |= 4; break; }
            for (int64_t k = 0; k < ef; k++) {
                P.dsk[K - 1] = hds[k];
                P.vpar[K] = hv[k]; P.b[K] = hb[k];
                P.ca[K] = hca[k]; P.cb[K] = hcb[k]; P.w[K] = hw[k];
                for (int l = 0; l < nl; l++) { P.eta[l * P.cap + K] = heta[l * ecap + k]; P.chi[l * P.cap + K] = hchi[l * ecap + k]; }
                K++;
            }
            P.K = K;
            for (int l = 0; l < nl; l++) {
                double nu_l = line_nu(m, l);
                for (int q = 0; q < Q; q++) {
                    double aq = m->roots[q] * bo;        /* r_q b_o */
                    double chi_lo = 0.0, eta_lo = 0.0;   /* line l's own share at the origin */
                    for (int64_t k = 0; k < K; k++) {
                        double v = P.vpar[k], bk = P.b[k];
                        double ch = 0.0, et = 0.0;
                        for (int l2 = 0; l2 < nl; l2++) {
                            double nu2 = line_nu(m, l2);
                            double x = (C_LIGHT * (nu_l - nu2) / nu2 + (nu_l / nu2) * (aq * (1.0 - v / C_LIGHT) - v)) / bk;
                            double dnu = nu2 * bk / C_LIGHT;
                            double phi = exp(-x * x) / (dnu * SQRT_PI);
                            ch += P.chi[l2 * P.cap + k] * phi;
                            et += P.eta[l2 * P.cap + k] * phi;
                            if (k == P.ko && l2 == l) {
                                chi_lo = P.chi[l2 * P.cap + k] * phi;
                                eta_lo = P.eta[l2 * P.cap + k] * phi;
                            }
                            if (l2 == l) phil[k] = phi;
                        }
                        if (chi_sca) {
                            /* isotropic coherent scattering (Sec. 3.3, eq. 'GFE' with Psi- = 0):
                             * opacity chi_sca, emissivity chi_sca J at the comoving frequency,
                             * both interpolated between the point's cells */
                            double wk = P.w[k];
                            double r = (aq * (1.0 - v / C_LIGHT) - v) / bk;
                            double xs = (1.0 - wk) * chi_sca[P.ca[k]] + wk * chi_sca[P.cb[k]];
                            double Jk = (1.0 - wk) * spectrum_at(m, Jsca, P.ca[k], l, r) +
                                        wk * spectrum_at(m, Jsca, P.cb[k], l, r);
                            ch += xs;
                            et += xs * Jk;
                        }
                        if (ch < m->chi_min) ch = m->chi_min;
                        chi[k] = ch; eta[k] = et; S[k] = et / ch;
                    }
                    for (int64_t k = 0; k + 1 < K; k++) {
                        double dt = 0.5 * (chi[k] + chi[k + 1]) * P.dsk[k];
                        dtau[k] = dt < m->dtau_min ? m->dtau_min : dt;
                    }
                    /* incoming CMB at both ends, at the comoving frequency there */
                    double nu_o = nu_l * (1.0 + aq / C_LIGHT);
                    double I0 = planck(nu_o * (1.0 - P.vpar[0] / C_LIGHT), m->T_cmb);
                    double IK = planck(nu_o * (1.0 - P.vpar[K - 1] / C_LIGHT), m->T_cmb);
                    double u, lam;
                    or_feautrier(K, P.ko, dtau, S, I0, IK, &u, &lam, work);
                    double w = m->weights[q];
                    accJ[l] += w * u;
                    accL[l] += w * lam * chi_lo / chi[P.ko];
                    accE[l] += w * (u - lam * eta_lo / chi[P.ko]);
                    accN[l * Q + q] += u;
                    if (band > 0) {
                        /* band of row ko of the inverse (Sec. 3.4): the points ko -+ j of the
                         * backward (ray pb) and forward (ray pf) halves, j = 1..band (none
                         * for an isolated origin, K = 1) */
                        if (K > 1) or_feautrier_band(K, P.ko, band, dtau, xrow, rwork);
                        double jb = u - lam * eta_lo / chi[P.ko];
                        for (int j = 1; j <= band; j++) {
                            for (int side = 0; side < 2 && K > 1; side++) {
                                int64_t k = side == 0 ? P.ko - j : P.ko + j;
                                if (k < 0 || k >= K) continue;
                                int r = side == 0 ? pb[p] : pf[p];
                                double eta_l = P.eta[l * P.cap + k] * phil[k];
                                jb -= xrow[k] * eta_l / chi[k];
                                accM[((size_t)l * R + r) * band + (j - 1)] +=
                                    w * xrow[k] * chi_c[l * N + o] * phil[k] / chi[k];
                            }
                            accEb[(j - 1) * nl + l] += w * jb;
                        }
                    }
                }
            }
        }
        for (int l = 0; l < nl; l++) {
            J[io * nl + l] = accJ[l] / npairs;
            L[io * nl + l] = accL[l] / npairs;
            Jeff[io * nl + l] = accE[l] / npairs;
            if (Jnu) for (int q = 0; q < Q; q++) Jnu[(io * nl + l) * Q + q] = accN[l * Q + q] / npairs;
            for (int j = 0; j < band; j++) {
                Jeffb[((size_t)j * n_orig + io) * nl + l] = accEb[j * nl + l] / npairs;
                for (int r = 0; r < R; r++)
                    Mb[(((size_t)io * nl + l) * R + r) * band + j] = accM[((size_t)l * R + r) * band + j] / npairs;
            }
        }
        free(cf); free(cb); free(nf); free(nb); free(dsf); free(dsb); free(vf); free(vb);
        free(hds); free(hv); free(hb); free(heta); free(hchi); pair_free(&P); free(hca); free(hcb); free(hw);
        free(chi); free(eta); free(S); free(dtau); free(work); free(accJ); free(accL); free(accE); free(accN);
        free(accEb); free(accM); free(xrow); free(rwork); free(phil);
    }
    free(eta_c); free(chi_c); free(pf); free(pb);
    return err ? -3 : 0;
}

int or_formal_solve(const or_model *m, const double *pops, int64_t n_orig, const int64_t *origins,
                    double *J, double *L, double *Jeff, double *Jnu, int nthreads) {
    return formal_solve_impl(m, pops, n_orig, origins, J, L, Jeff, Jnu, 0, NULL, NULL, NULL, NULL, nthreads);
}

/* Formal solution with isotropic, coherent scattering (Sec. 2.1 eq. 'RTE', Sec. 3.3 eq.
 * 'GFE'): a frequency-independent scattering opacity chi_sca[n] per cell, scattering
 * isotropically and without a change of frequency in the comoving frame. Then the
 * scattering opacity is the same up and down the ray (chi+ = chi_sca, chi- = 0), the
 * redistribution does not depend on the outgoing direction (Phi- = 0, so Psi- = 0), and
 * Psi+ = chi_sca J_nu: eq. 'GFE' for u is the second-order equation with opacity
 * chi + chi_sca and source (eta + chi_sca J)/(chi + chi_sca). As Sec. 3.3 prescribes, the
 * right-hand side is evaluated with the solution of the previous iteration: Jsca
 * [n][n_lines][Q] is the previous mean intensity of every cell in its own bins; at a
 * point of a ray it is read at the point's comoving offset from the line centre, in
 * units of the point's width, from the bins of the point's cells (spectrum_at),
 * interpolated between the cells like the line data. Jnu [n_orig][n_lines][Q] receives
 * the new one. Readings: the bins of line l carry the radiation scattered in line l's own
 * bins; chi_sca is interpolated like the line data at inserted points. */
int or_formal_solve_sca(const or_model *m, const double *pops, int64_t n_orig, const int64_t *origins,
                        const double *chi_sca, const double *Jsca, double *J, double *L, double *Jeff, double *Jnu,
                        int nthreads) {
    return formal_solve_impl(m, pops, n_orig, origins, J, L, Jeff, Jnu, 0, NULL, NULL, chi_sca, Jsca, nthreads);
}

/* Formal solution with the band-diagonal ALO of Sec. 3.4 (eq. 'ALO', 'ourJeff'): besides
 * J, L (diagonal) and Jeff (bandwidth 0), for bandwidth b = 1..band
 *   Jeffb[b-1][io][l] = (1/P) sum_p sum_q w_q (u - sum_{|k-ko|<=b} (T^-1)_{ko,k} eta_l(k)/chi(k)),
 * and per half-ray r and band slot j (the j-th point of the half from the origin)
 *   Mb[io][l][r][j-1] = (1/P) sum_q w_q (T^-1)_{ko,k} chi_int,l(o) phi_l(k)/chi(k),
 * the weight with which A_ul n_u at that point enters the rate equation of the origin
 * (eq. 'ourALI' with the operator of eq. 'ALO': the emissivity at point k is
 * h nu/4pi A n_u(k) phi_l(k), the prefactor is chi_int,l(o) = h nu/4pi (n_l B_lu - n_u B_ul)
 * at the origin, from the old populations). */
int or_formal_solve_band(const or_model *m, const double *pops, int64_t n_orig, const int64_t *origins, int band,
                         double *J, double *L, double *Jeff, double *Jeffb, double *Mb, int nthreads) {
    if (band < 1) return -1;
    return formal_solve_impl(m, pops, n_orig, origins, J, L, Jeff, NULL, band, Jeffb, Mb, NULL, NULL, nthreads);
}

/* Cells behind band slot j (1..band) of half-ray (o, r): the j-th expanded point from the
 * origin interpolates its line data between cells ca and cb with weight w on cb (w = 1 at
 * a traced cell); ca = cb = -1 where the half has fewer than j points. Outputs
 * [n_orig][R][band]. */
int or_band_geometry(const or_model *m, int64_t n_orig, const int64_t *origins, int band, int32_t *ca,
                     int32_t *cb, double *w) {
    int64_t cap = m->max_steps;
    int32_t *cells = malloc(sizeof(int32_t) * cap), *nsub = malloc(sizeof(int32_t) * cap);
    double *ds = malloc(sizeof(double) * cap), *vpar = malloc(sizeof(double) * cap);
    int err = (!cells || !nsub || !ds || !vpar);
    for (int64_t io = 0; io < n_orig && !err; io++) {
        int64_t o = origins[io];
        for (int r = 0; r < m->R && !err; r++) {
            int64_t len; int de;
            if (or_trace(m, o, r, cap, cells, nsub, ds, vpar, &len, &de)) { err = 1; break; }
            for (int j = 1; j <= band; j++) {
                size_t k = ((size_t)io * m->R + r) * band + (j - 1);
                ca[k] = -1; cb[k] = -1; w[k] = 0.0;
                /* walk the expanded points: element e holds nsub[e] + 1 points, the last
                 * one its own cell; point x of element e is sub-point x - x0 + 1 */
                int64_t x0 = 0, prev = o;
                for (int64_t e = 0; e < len; e++) {
                    int64_t cnt = nsub[e] + 1;
                    if (j - 1 < x0 + cnt) {
                        ca[k] = (int32_t)prev;
                        cb[k] = cells[e];
                        w[k] = (double)(j - x0) / (double)cnt;
                        break;
                    }
                    x0 += cnt;
                    prev = cells[e];
                }
            }
        }
    }
    free(cells); free(nsub); free(ds); free(vpar);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------ statistical equilibrium */

/* Collisional de-excitation coefficient of pair (i>j) at temperature T: linear
 * interpolation in T on the tabulated grid, constant beyond its ends (Reading). */
static double k_down(const or_model *m, int i, int j, double T) {
    int pair = i * (i - 1) / 2 + j;
    const double *k = &m->K_down[pair * m->n_T];
    const double *Tg = m->T_grid;
    if (m->n_T == 1 || T <= Tg[0]) return k[0];
    if (T >= Tg[m->n_T - 1]) return k[m->n_T - 1];
    int a = 0;
    while (Tg[a + 1] < T) a++;
    double t = (T - Tg[a]) / (Tg[a + 1] - Tg[a]);
    return k[a] + t * (k[a + 1] - k[a]);
}

/* Rate generator of cell c (eq. 'ourALI'): G[i*n+j] = rate j->i for i != j and
 * G[j*n+j] = -sum_i rate j->i, with u->l = A_ul oml_l + B_ul Jeff_l + C_ul and
 * l->u = B_lu Jeff_l + C_lu for every line, where oml_l is the factor left of the
 * spontaneous rate by the ALO (1 - L with the diagonal ALO), and all collisional pairs
 * C_ij = K_ij(T) n_coll with excitation by detailed balance.
 * Reading: the paper prints the excitation factor exp(+h nu/kT); the physical form
 * C_lu = C_ul (g_u/g_l) exp(-(E_u - E_l)/kT) is used, the only one that makes high
 * densities thermalise to LTE. */
int or_cell_generator(const or_model *m, int64_t c, const double *oml, const double *Ec, double *G) {
    int n = m->n_lev;
    double P[64 * 64];
    if (n > 64) return -1;
    memset(P, 0, sizeof(double) * n * n);
    for (int l = 0; l < m->n_lines; l++) {
        int u = m->up[l], lo = m->lo[l];
        double Bul, Blu;
        einstein_b(m, l, &Bul, &Blu);
        P[u * n + lo] += m->A[l] * oml[l] + Bul * Ec[l];
        P[lo * n + u] += Blu * Ec[l];
    }
    double T = m->T[c];
    for (int i = 1; i < n; i++)
        for (int j = 0; j < i; j++) {
            double Cd = k_down(m, i, j, T) * m->n_coll[c];
            double Cu = Cd * m->g[i] / m->g[j] * exp(-(m->E[i] - m->E[j]) / (K_BOLTZ * T));
            P[i * n + j] += Cd;
            P[j * n + i] += Cu;
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) G[i * n + j] = 0.0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            if (i == j) continue;
            G[i * n + j] += P[j * n + i];
            G[j * n + j] -= P[j * n + i];
        }
    return 0;
}

/* Double-double numbers (hi + lo, |lo| <= ulp(hi)/2) from error-free transformations
 * (Knuth's TwoSum, the fused multiply-add for the product's error; Dekker 1971): about
 * 106 bits of mantissa, enough to resolve levels whose populations span thirty decades. */
typedef struct { double hi, lo; } dd;
static dd dd_from(double a) { dd r = {a, 0.0}; return r; }
static dd dd_norm(double s, double e) { double h = s + e; dd r = {h, e - (h - s)}; return r; }
static dd dd_add(dd a, dd b) {
    double s = a.hi + b.hi, bb = s - a.hi, e = (a.hi - (s - bb)) + (b.hi - bb);
    return dd_norm(s, e + a.lo + b.lo);
}
static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi, e = fma(a.hi, b.hi, -p);
    return dd_norm(p, e + (a.hi * b.lo + a.lo * b.hi));
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(dd_from(q1), b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(dd_from(q2), b));
    double q3 = r.hi / b.hi;
    return dd_add(dd_norm(q1, q2), dd_from(q3));
}

/* Gaussian elimination with partial pivoting in double-double arithmetic (in place). */
static int lu_solve_dd(int n, dd *M, dd *b) {
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++) if (fabs(M[r * n + c].hi) > fabs(M[piv * n + c].hi)) piv = r;
        if (M[piv * n + c].hi == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; k++) { dd t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t; }
            dd t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            dd f = dd_div(M[r * n + c], M[c * n + c]);
            for (int k = c; k < n; k++) M[r * n + k] = dd_sub(M[r * n + k], dd_mul(f, M[c * n + k]));
            b[r] = dd_sub(b[r], dd_mul(f, b[c]));
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        dd s = b[r];
        for (int k = r + 1; k < n; k++) s = dd_sub(s, dd_mul(M[r * n + k], b[k]));
        b[r] = dd_div(s, M[r * n + r]);
    }
    return 0;
}

/* Statistical equilibrium of one cell with the diagonal ALO (eq. 'ourALI'), rates as in
 * or_cell_generator with oml = 1 - L. The last equation is replaced by
 * sum_i n_i = n_spec (Reading). The system is solved by LU with partial pivoting in
 * double-double arithmetic, the diagonal formed from the exit rates in the same
 * arithmetic: in FP64 a 20-level rotor's populations lose up to seven digits (those
 * holding 1e-7 of the cell off by 20%, and rounding-level negative values near 1e-30
 * that would trip the validity check); the rates themselves are the FP64 values of
 * or_cell_generator. */
static int stateq_cell(const or_model *m, int64_t c, const double *Jc, const double *Lc,
                       const double *Ec, double *out) {
    int n = m->n_lev;
    double G[64 * 64], oml[64 * 64];
    dd M[64 * 64], b[64];
    if (n > 64 || m->n_lines > 64 * 64) return -1;
    (void)Jc;
    for (int l = 0; l < m->n_lines; l++) oml[l] = 1.0 - Lc[l];
    if (or_cell_generator(m, c, oml, Ec, G)) return -1;
    /* off-diagonal rates as they are; each diagonal entry the double-double sum of its
     * column's exit rates, so that the columns sum to zero to ~1e-32 (an FP64 diagonal
     * leaves ~1e-16 of the largest flux unbalanced, which swamps levels near 1e-30) */
    for (int j = 0; j < n; j++) {
        dd d = dd_from(0.0);
        for (int i = 0; i < n; i++) {
            if (i == j) continue;
            M[i * n + j] = dd_from(G[i * n + j]);
            d = dd_sub(d, M[i * n + j]);
        }
        M[j * n + j] = d;
    }
    for (int j = 0; j < n; j++) { M[(n - 1) * n + j] = dd_from(1.0); b[j] = dd_from(0.0); }
    b[n - 1] = dd_from(m->n_spec[c]);
    if (lu_solve_dd(n, M, b)) return -2;
    for (int i = 0; i < n; i++) out[i] = b[i].hi + b[i].lo;
    return 0;
}

/* Level populations of all cells from J, L, Jeff ([n][n_lines]). Validity check
 * (Sec. 6.1): a cell whose populations come out negative (below -1e-28 of the cell) or
 * non-finite is solved again with part of the ALO removed; here the diagonal ALO is
 * dropped (L = 0, Jeff = J).
 * Returns the number of such cells in *n_fallback. */
int or_stateq(const or_model *m, const double *J, const double *L, const double *Jeff,
              double *pops_out, int64_t *n_fallback) {
    int nl = m->n_lines, n = m->n_lev;
    int64_t nf = 0;
    double zeros[64];
    for (int l = 0; l < 64; l++) zeros[l] = 0.0;
    for (int64_t c = 0; c < m->n; c++) {
        double *out = &pops_out[c * n];
        int rc = stateq_cell(m, c, &J[c * nl], &L[c * nl], &Jeff[c * nl], out);
        int bad = rc != 0;
        /* Reading: a value above -1e-28 of the cell is rounding noise of the solve (its
         * resolution is ~1e-32 of the cell), not an unphysical population */
        for (int i = 0; i < n && !bad; i++) if (!(out[i] >= -1e-28 * m->n_spec[c]) || !isfinite(out[i])) bad = 1;
        if (bad) {
            nf++;
            if (stateq_cell(m, c, &J[c * nl], zeros, &J[c * nl], out)) return -1;
        }
    }
    *n_fallback = nf;
    return 0;
}

/* Maximum relative change over cells and levels with n_i/n_spec >= 1e-10 (Reading: the
 * paper quotes the relative change in level populations without naming the norm). */
double or_max_rel_change(const or_model *m, const double *old, const double *new_) {
    double mx = 0.0;
    for (int64_t c = 0; c < m->n; c++)
        for (int i = 0; i < m->n_lev; i++) {
            double a = new_[c * m->n_lev + i], b = old[c * m->n_lev + i];
            if (a < 1e-10 * m->n_spec[c]) continue;
            double d = fabs(a - b) / a;
            if (d > mx) mx = d;
        }
    return mx;
}

/* Ng acceleration (Sec. 3.4; Ng 1974, Olson et al. 1986) from four iterates x0 (newest)
 * .. x3 with differences D_i = x_i - x_{i+1}: minimise |D0 - a1 (D0-D1) - a2 (D0-D2)|^2
 * with uniform weights, then x = (1-a1-a2) x0 + a1 x1 + a2 x2. Returns -1 if the
 * normal equations are singular. */
int or_ng(int64_t n, const double *x0, const double *x1, const double *x2, const double *x3,
          double *out) {
    double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
    for (int64_t k = 0; k < n; k++) {
        double D0 = x0[k] - x1[k], D1 = x1[k] - x2[k], D2 = x2[k] - x3[k];
        double Q1 = D0 - D1, Q2 = D0 - D2;
        a11 += Q1 * Q1; a12 += Q1 * Q2; a22 += Q2 * Q2;
        b1 += Q1 * D0; b2 += Q2 * D0;
    }
    double det = a11 * a22 - a12 * a12;
    if (det == 0.0 || !isfinite(det)) return -1;
    double a1 = (b1 * a22 - b2 * a12) / det;
    double a2 = (a11 * b2 - a12 * b1) / det;
    for (int64_t k = 0; k < n; k++) out[k] = (1.0 - a1 - a2) * x0[k] + a1 * x1[k] + a2 * x2[k];
    return 0;
}

/* Accelerated Lambda iteration (Sec. 2.2.1, 3.4): formal solve -> statistical
 * equilibrium -> convergence check, optionally with an Ng step every ng_period
 * iterations on the fractional populations n_i/n_spec (Reading: "uniform weighting" is
 * taken over levels of the fractional populations). pops holds the start and receives
 * the result. changes[it] gets each iteration's max relative change. Returns the
 * number of iterations, negative on error; *converged is set when change < tol. */
int or_ali(const or_model *m, double *pops, double tol, int max_iter, int ng_period,
           double *changes, int *converged, int nthreads) {
    int64_t N = m->n, nl = m->n_lines, nv = m->n * m->n_lev;
    double *J = malloc(sizeof(double) * N * nl), *L = malloc(sizeof(double) * N * nl);
    double *E = malloc(sizeof(double) * N * nl), *nw = malloc(sizeof(double) * nv);
    double *hist[4];
    for (int i = 0; i < 4; i++) hist[i] = malloc(sizeof(double) * nv);
    double *ng_out = malloc(sizeof(double) * nv);
    int64_t *orig = malloc(sizeof(int64_t) * N);
    for (int64_t c = 0; c < N; c++) orig[c] = c;
    int nh = 0, it = 0;
    *converged = 0;
    for (it = 0; it < max_iter; it++) {
        if (or_formal_solve(m, pops, N, orig, J, L, E, NULL, nthreads)) { it = -1; break; }
        int64_t nf;
        if (or_stateq(m, J, L, E, nw, &nf)) { it = -2; break; }
        double ch = or_max_rel_change(m, pops, nw);
        changes[it] = ch;
        memcpy(pops, nw, sizeof(double) * nv);
        if (ch < tol) { *converged = 1; it++; break; }
        if (ng_period > 0) {
            double *t = hist[3]; hist[3] = hist[2]; hist[2] = hist[1]; hist[1] = hist[0]; hist[0] = t;
            for (int64_t c = 0; c < N; c++)
                for (int i = 0; i < m->n_lev; i++) hist[0][c * m->n_lev + i] = pops[c * m->n_lev + i] / m->n_spec[c];
            if (nh < 4) nh++;
            if (nh == 4 && (it + 1) % ng_period == 0) {
                if (or_ng(nv, hist[0], hist[1], hist[2], hist[3], ng_out) == 0) {
                    int ok = 1;
                    for (int64_t k = 0; k < nv; k++) if (!(ng_out[k] >= 0.0)) { ok = 0; break; }
                    if (ok)
                        for (int64_t c = 0; c < N; c++)
                            for (int i = 0; i < m->n_lev; i++)
                                pops[c * m->n_lev + i] = ng_out[c * m->n_lev + i] * m->n_spec[c];
                }
                nh = 0;
            }
        }
    }
    free(J); free(L); free(E); free(nw); free(ng_out); free(orig);
    for (int i = 0; i < 4; i++) free(hist[i]);
    return it;
}

/* All half-rays of a list of origins, in CSR form by (origin, ray): first call with
 * cells == NULL to get the counts in len[n_orig * R]; second call fills cells, nsub, ds,
 * vpar at offsets off[n_orig * R] (exclusive prefix sums of len). dead[n_orig * R] flags
 * dead ends. */
int or_trace_all(const or_model *m, int64_t n_orig, const int64_t *origins, const int64_t *off,
                 int32_t *len, int32_t *cells, int32_t *nsub, double *ds, double *vpar, uint8_t *dead,
                 int nthreads) {
    int err = 0;
    int64_t cap = m->max_steps;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 16) reduction(|:err)
#endif
    for (int64_t io = 0; io < n_orig; io++) {
        int32_t *c = malloc(sizeof(int32_t) * cap), *ns = malloc(sizeof(int32_t) * cap);
        double *d = malloc(sizeof(double) * cap), *v = malloc(sizeof(double) * cap);
        for (int r = 0; r < m->R; r++) {
            int64_t ln; int de;
            if (or_trace(m, origins[io], r, cap, c, ns, d, v, &ln, &de)) { err = 1; continue; }
            int64_t k = io * m->R + r;
            if (!cells) { len[k] = (int32_t)ln; if (dead) dead[k] = (uint8_t)de; continue; }
            memcpy(cells + off[k], c, sizeof(int32_t) * ln);
            memcpy(nsub + off[k], ns, sizeof(int32_t) * ln);
            memcpy(ds + off[k], d, sizeof(double) * ln);
            memcpy(vpar + off[k], v, sizeof(double) * ln);
        }
        free(c); free(ns); free(d); free(v);
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------ imaging */

/* Formal solution of the first-order transfer equation dI/dtau = S - I across one
 * interval of optical depth d, with S linear in tau between its end values Sa (entry)
 * and Sb (exit) (Olson & Kunasz 1987):
 *   I_out = e I_in + (alpha - e) Sa + (1 - alpha) Sb,  e = exp(-d), alpha = (1 - e)/d.
 * Reading: for d < 1e-3 the two weights are taken from their Taylor series,
 *   1 - alpha = d/2 - d^2/6 + d^3/24 - d^4/120,  alpha - e = d/2 - d^2/3 + d^3/8 - d^4/30,
 * because 1 - alpha cancels there and a floored opacity makes S as large as eta/chi_min. */
double or_linear_source_step(double I_in, double d, double Sa, double Sb) {
    double e = exp(-d), wa, wb;
    if (d < 1e-3) {
        wb = d * (0.5 - d * (1.0 / 6.0 - d * (1.0 / 24.0 - d / 120.0)));
        wa = d * (0.5 - d * (1.0 / 3.0 - d * (1.0 / 8.0 - d / 30.0)));
    } else {
        double alpha = -expm1(-d) / d;
        wb = 1.0 - alpha;
        wa = alpha - e;
    }
    return e * I_in + wa * Sa + wb * Sb;
}

/* Outward intensity after K points with increments dtau[0..K-2] and source S[0..K-1],
 * entering with I0 at point 0. */
double or_first_order(int64_t K, const double *dtau, const double *S, double I0) {
    double I = I0;
    for (int64_t k = 0; k + 1 < K; k++) I = or_linear_source_step(I, dtau[k], S[k], S[k + 1]);
    return I;
}

/* Image of the model along ray direction r (Sec. 3.5, 'Imaging the model'): every
 * origin point o gives one image point, the projection of its position on the plane
 * orthogonal to n = dirs[r], with the intensity leaving the model along n on the ray
 * pair through o. xy[o] = (x.e1, x.e2) with e1 = (z x n)/|z x n| (x in place of z when
 * |n_z| >= 0.9) and e2 = n x e1.
 * Readings (the paper says only that images come from the outward radiation at the
 * ray-pair end points):
 *  - channel c has frequency nu_l (1 + u_c/c) in the rest frame of the model (u_c in
 *    velocity units, as the bins' r_q b_o); at a point of velocity v its comoving
 *    frequency is nu (1 - n.v/c), to first order in v/c, for radiation travelling
 *    along n; all lines contribute to opacity and emissivity as in the formal solve;
 *  - the points, path lengths, interpolation, floors and dtau are those of the formal
 *    solve's ray pair (the far end of the half-ray along -n first);
 *  - the intensity is carried along n with the first-order linear-source step above,
 *    entering with the CMB at the comoving frequency of the far end of the -n half;
 *    a model point with both halves empty shows the CMB at its own comoving frequency.
 * Output I[io][n_ch]. */
int or_image(const or_model *m, const double *pops, int r, int line, int n_ch, const double *u_ch,
             int64_t n_orig, const int64_t *origins, double *I, double *xy, int nthreads) {
    if (r < 0 || r >= m->R || line < 0 || line >= m->n_lines || n_ch < 1) return -1;
    int nl = m->n_lines;
    int64_t N = m->n;
    const double *n = &m->dirs[3 * r];
    int rb = m->antipode[r];
    double e1[3], e2[3];
    {
        double a[3] = {0.0, 0.0, 1.0};
        if (fabs(n[2]) >= 0.9) { a[0] = 1.0; a[2] = 0.0; }
        e1[0] = a[1] * n[2] - a[2] * n[1];
        e1[1] = a[2] * n[0] - a[0] * n[2];
        e1[2] = a[0] * n[1] - a[1] * n[0];
        double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int i = 0; i < 3; i++) e1[i] /= l1;
        e2[0] = n[1] * e1[2] - n[2] * e1[1];
        e2[1] = n[2] * e1[0] - n[0] * e1[2];
        e2[2] = n[0] * e1[1] - n[1] * e1[0];
    }
    double *eta_c = malloc(sizeof(double) * N * nl), *chi_c = malloc(sizeof(double) * N * nl);
    if (!eta_c || !chi_c) { free(eta_c); free(chi_c); return -2; }
    all_line_integrals(m, pops, eta_c, chi_c);
    double nu_l = line_nu(m, line);
    int err = 0;
    int64_t cap = m->max_steps;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 4) reduction(|:err)
#endif
    for (int64_t io = 0; io < n_orig; io++) {
        int64_t o = origins[io];
        const double *x = &m->pos[3 * o];
        if (xy) {
            xy[2 * io] = x[0] * e1[0] + x[1] * e1[1] + x[2] * e1[2];
            xy[2 * io + 1] = x[0] * e2[0] + x[1] * e2[1] + x[2] * e2[2];
        }
        int32_t *cf = malloc(sizeof(int32_t) * cap), *cb = malloc(sizeof(int32_t) * cap);
        int32_t *nf = malloc(sizeof(int32_t) * cap), *nb = malloc(sizeof(int32_t) * cap);
        double *dsf = malloc(sizeof(double) * cap), *dsb = malloc(sizeof(double) * cap);
        double *vf = malloc(sizeof(double) * cap), *vb = malloc(sizeof(double) * cap);
        double *buf = NULL;
        do {
            if (!cf || !cb || !nf || !nb || !dsf || !dsb || !vf || !vb) { err |= 1; break; }
            int64_t lf, lb; int de;
            if (or_trace(m, o, r, cap, cf, nf, dsf, vf, &lf, &de)) { err |= 2; break; }
            if (or_trace(m, o, rb, cap, cb, nb, dsb, vb, &lb, &de)) { err |= 2; break; }
            int64_t Kb = 0, Kf = 0;
            for (int64_t e = 0; e < lb; e++) Kb += nb[e] + 1;
            for (int64_t e = 0; e < lf; e++) Kf += nf[e] + 1;
            int64_t K = Kb + 1 + Kf;
            /* per point: path length to the next point, rest-frame line-of-sight velocity
             * n.v, width, line data; then per channel chi, S and dtau */
            buf = malloc(sizeof(double) * ((size_t)K * (6 + 2 * (size_t)nl) + 2 * (size_t)K));
            if (!buf) { err |= 1; break; }
            double *ds = buf, *w = ds + K, *b = w + K, *eta = b + K, *chi = eta + K * nl;
            double *ch = chi + K * nl, *S = ch + K, *dtau = S + K, *tmp = dtau + K;
            double *hds = tmp, *hv = tmp + K;   /* scratch for one expanded half (reused) */
            double *hb = malloc(sizeof(double) * K * (1 + 2 * (size_t)nl));
            if (!hb) { err |= 1; break; }
            double *heta = hb + K, *hchi = heta + K * nl;
            double nvo = n[0] * m->vel[3 * o] + n[1] * m->vel[3 * o + 1] + n[2] * m->vel[3 * o + 2];
            /* the -n half, far end first: its line-of-sight velocity is (-n).(v - v_o) */
            int64_t eb = expand_half(m, o, lb, cb, nb, dsb, vb, eta_c, chi_c, hds, hv, hb, heta, hchi, K, K, NULL, NULL, NULL);
            int64_t k = 0;
            for (int64_t j = eb - 1; j >= 0; j--, k++) {
                ds[k] = hds[j];
                w[k] = nvo - hv[j];
                b[k] = hb[j];
                for (int l = 0; l < nl; l++) { eta[l * K + k] = heta[l * K + j]; chi[l * K + k] = hchi[l * K + j]; }
            }
            ds[k] = 0.0; w[k] = nvo; b[k] = or_width(m, o);
            for (int l = 0; l < nl; l++) { eta[l * K + k] = eta_c[l * N + o]; chi[l * K + k] = chi_c[l * N + o]; }
            k++;
            int64_t ef = expand_half(m, o, lf, cf, nf, dsf, vf, eta_c, chi_c, hds, hv, hb, heta, hchi, K, K, NULL, NULL, NULL);
            for (int64_t j = 0; j < ef; j++, k++) {
                ds[k - 1] = hds[j];
                w[k] = nvo + hv[j];
                b[k] = hb[j];
                for (int l = 0; l < nl; l++) { eta[l * K + k] = heta[l * K + j]; chi[l * K + k] = hchi[l * K + j]; }
            }
            for (int c = 0; c < n_ch; c++) {
                double u = u_ch[c];
                for (int64_t q = 0; q < K; q++) {
                    double x_ch = 0.0, x_et = 0.0;
                    for (int l2 = 0; l2 < nl; l2++) {
                        double nu2 = line_nu(m, l2);
                        double xx = (C_LIGHT * (nu_l - nu2) / nu2 + (nu_l / nu2) * (u * (1.0 - w[q] / C_LIGHT) - w[q])) / b[q];
                        double dnu = nu2 * b[q] / C_LIGHT;
                        double phi = exp(-xx * xx) / (dnu * SQRT_PI);
                        x_ch += chi[l2 * K + q] * phi;
                        x_et += eta[l2 * K + q] * phi;
                    }
                    if (x_ch < m->chi_min) x_ch = m->chi_min;
                    ch[q] = x_ch;
                    S[q] = x_et / x_ch;
                }
                for (int64_t q = 0; q + 1 < K; q++) {
                    double dt = 0.5 * (ch[q] + ch[q + 1]) * ds[q];
                    dtau[q] = dt < m->dtau_min ? m->dtau_min : dt;
                }
                double nu_c = nu_l * (1.0 + u / C_LIGHT);
                double I0 = planck(nu_c * (1.0 - w[0] / C_LIGHT), m->T_cmb);
                I[io * n_ch + c] = or_first_order(K, dtau, S, I0);
            }
            free(hb);
        } while (0);
        free(cf); free(cb); free(nf); free(nb); free(dsf); free(dsb); free(vf); free(vb); free(buf);
    }
    free(eta_c); free(chi_c);
    return err ? -3 : 0;
}
