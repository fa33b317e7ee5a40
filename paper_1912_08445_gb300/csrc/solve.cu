// K2 (line data) and K3 (Feautrier formal solve with the diagonal ALO), Sec. 3.3-3.4.
#include <cmath>
#include "common.cuh"

using namespace mg;

namespace {

// ---------------------------------------------------------------- K2 line data
// eta_int = h nu/4pi n_u A_ul, chi_int = h nu/4pi (n_l B_lu - n_u B_ul) (eq. 'lines'),
// stored per point as [L][2] so that one gather brings all lines of a point.
__global__ void k_line_data(int64_t n, int L, int nlev, const double *__restrict__ pops,
                            const LineConst *__restrict__ lc, double *__restrict__ line, float *__restrict__ linef, unsigned long long *neg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * L) return;
    const int64_t c = t / L;
    const int l = (int)(t - c * L);
    const LineConst k = lc[l];
    const double nu_ = pops[c * nlev + k.up], nl_ = pops[c * nlev + k.lo];
    const double eta = k.pre * nu_ * k.A;
    const double chi = k.pre * (nl_ * k.Blu - nu_ * k.Bul);
    line[2 * t] = eta;
    line[2 * t + 1] = chi;
    if (chi < 0.0) atomicAdd(neg, 1ull);
    if (linef) {
        linef[2 * t] = (float)eta;
        linef[2 * t + 1] = (float)chi;
    }
}

struct SolveArgs {
    int64_t n;
    int32_t R, P, L, Q;
    const int32_t *pf, *pb;
    const int64_t *ray_off;
    const int32_t *cells, *xcum;
    const double *ds, *vpar;
    const double *b;
    const double *line;
    const LineConst *lc;
    const double *roots, *weights;
    const int32_t *ovl_off;
    const Overlap *ovl;
    double chi_min, dtau_min, T_cmb;
    double *J, *Lout, *Jeff, *Lc, *Jnu;
    int32_t kmax;
    int32_t *err;
    const int32_t *olist;    // optional list of origins (FP64 promotion), count in *ocount
    const int32_t *ocount;
    int32_t groups;          // FP64 kernel: warps that solve different ray pairs of a point (1: the whole CTA per pair)
    double *Jeffb;           // band ALO: [B][n][L] J_eff of bandwidths 1..B
    double *Mb;              // band ALO: [n][L][R][B] coupling coefficients of the band points
    const double *chi_sca;   // scattering: [n] opacity, m^-1
    const double *Jsca;      // scattering: [n][L][Q] previous mean intensity per bin
};

__device__ __forceinline__ double planck_d(double nu, double T) {
    return 2.0 * kH * nu * nu * nu / (kC * kC) / expm1(kH * nu / (kKB * T));
}

// Stages the expanded points of half-ray (o, r) into the pair arrays: per point the path
// length to the neighbouring point towards the origin, the line-of-sight velocity, the
// width, and the two cells and weight that interpolate its line data (read from global
// memory during the sweep). Point x of the half (0 = nearest the origin) sits at pair
// index base + dir x; its path length goes to ds slot (dir < 0 ? idx : idx - 1).
struct PairSmem64 {
    double *ds, *v, *ib, *w;   // ib: 1/b, the reciprocal width (one division per point, not per bin)
    int32_t *ca, *cb;
};

// Threads tid = 0..nth-1 share the work.
__device__ void stage_half64(const SolveArgs &a, int64_t o, int r, int base, int dir, const PairSmem64 &S, int tid,
                             int nth) {
    const int64_t off = a.ray_off[o * a.R + r];
    const int len = (int)(a.ray_off[o * a.R + r + 1] - off);
    for (int e = tid; e < len; e += nth) {
        const int32_t c = a.cells[off + e];
        const int32_t prev = e ? a.cells[off + e - 1] : (int32_t)o;
        const int x0 = e ? a.xcum[off + e - 1] : 0;
        const int ns = a.xcum[off + e] - x0 - 1;
        const double pv = e ? a.vpar[off + e - 1] : 0.0;
        const double ve = a.vpar[off + e], dse = a.ds[off + e];
        const double bp = a.b[prev], bc = a.b[c];
        for (int j = 1; j <= ns + 1; j++) {
            const double w = (double)j / (double)(ns + 1);
            const int idx = base + dir * (x0 + j - 1);
            S.ds[dir < 0 ? idx : idx - 1] = dse / (double)(ns + 1);
            S.v[idx] = (1.0 - w) * pv + w * ve;
            S.ib[idx] = 1.0 / ((1.0 - w) * bp + w * bc);
            S.w[idx] = w;
            S.ca[idx] = prev;
            S.cb[idx] = c;
        }
    }
}

// Opacity, emissivity and line l's own share at pair point k for bin (l, q), and line l's
// own profile phi_l there.
struct Pt64 {
    double chi, eta, chil, etal, phil;
};

// Mean intensity of cell c in the bins of line l at offset r (in widths) from the line
// centre: linear interpolation between the Gauss-Hermite roots (ascending), the outermost
// values beyond them (binary search for the bracketing roots).
__device__ __forceinline__ double spectrum_at(const SolveArgs &a, int64_t c, int l, double r) {
    const double *Jc = a.Jsca + ((size_t)c * a.L + l) * a.Q;
    const double *x = a.roots;
    const int Q = a.Q;
    if (Q == 1 || r <= x[0]) return Jc[0];
    if (r >= x[Q - 1]) return Jc[Q - 1];
    int lo = 0, hi = Q - 1;   // x[lo] <= r < x[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x[mid] <= r) lo = mid;
        else hi = mid;
    }
    const double t = (r - x[lo]) / (x[lo + 1] - x[lo]);
    return Jc[lo] + t * (Jc[lo + 1] - Jc[lo]);
}

// k1 = 1 + a_q/c: the comoving shift a_q (1 - v/c) - v is a_q - v k1 (no division).
// SCAT: isotropic coherent scattering adds chi_sca to the opacity and chi_sca J to the
// emissivity (Sec. 3.3, eq. 'GFE' with Psi+ = chi_sca J and Psi- = 0), both interpolated
// between the point's cells, J read at the point's comoving offset from the line centre.
template <bool SCAT = false>
__device__ __forceinline__ Pt64 point64(const SolveArgs &a, int l, double aq, double k1, int k, const PairSmem64 &S) {
    constexpr double kCsp = kC / kSqrtPi;
    const double v = S.v[k], ibk = S.ib[k], w = S.w[k];
    const double *pa = a.line + (int64_t)S.ca[k] * 2 * a.L, *pb = a.line + (int64_t)S.cb[k] * 2 * a.L;
    Pt64 p{0.0, 0.0, 0.0, 0.0, 0.0};
    const int o0 = a.ovl_off[l], o1 = a.ovl_off[l + 1];
    const double base = aq - v * k1;
    for (int i = o0; i < o1; i++) {
        const Overlap ov = a.ovl[i];
        const double x = (ov.dnl + ov.rat * base) * ibk;
        const double phi = exp(-x * x) * (ov.inv_nu2 * ibk) * kCsp;
        const double et = ((1.0 - w) * pa[2 * ov.l2] + w * pb[2 * ov.l2]) * phi;
        const double ch = ((1.0 - w) * pa[2 * ov.l2 + 1] + w * pb[2 * ov.l2 + 1]) * phi;
        p.eta += et;
        p.chi += ch;
        if (i == o0) { p.etal = et; p.chil = ch; p.phil = phi; }
    }
    if constexpr (SCAT) {
        const int64_t ca = S.ca[k], cb = S.cb[k];
        const double r = base * ibk;
        const double xs = (1.0 - w) * a.chi_sca[ca] + w * a.chi_sca[cb];
        const double Jk = (1.0 - w) * spectrum_at(a, ca, l, r) + w * spectrum_at(a, cb, l, r);
        p.chi += xs;
        p.eta += xs * Jk;
    }
    return p;
}

// One CTA per origin point; the CTA (or, for few bins, each of its warps) loops over the
// ray pairs, staging each expanded pair in shared memory, and each thread solves its
// frequency bins.
//
// Sweep in rescaled Rybicki-Hummer variables from a far end towards the origin: with
// dtau_k between points k and k+1, F_k = dtau_k Phi_k and z_k = dtau_k psi_k,
//   boundary row:  Phi_0 = dtau_0/2 + 1,              psi_0 = (dtau_0 S_0/2 + I) iota_0,
//   interior row:  Phi_k = t_k + Phi_{k-1} iota_{k-1}, psi_k = (t_k S_k + psi_{k-1}) iota_k,
//   with t_k = (dtau_{k-1} + dtau_k)/2 and iota_k = 1/(1 + dtau_k Phi_k).
// At the origin, with sigma = 2/(dtau_- + dtau_+):
//   D = 1 + sigma (Phi_b iota_b + Phi_f iota_f),  Lambda*_oo = 1/D,
//   u - Lambda* S_o = sigma (psi_b + psi_f)/D,    1 - Lambda* = sigma (Phi_b iota_b + Phi_f iota_f)/D,
// all sums of non-negative terms. An empty half contributes Phi iota = 1, psi = I_o and
// dtau = 0 (the origin row is then the boundary row).
//
// Band-diagonal ALO (Sec. 3.4, eq. 'ALO'; B = bandwidth): with m the point next to the
// origin and m-1 the one before it, psi_m = g_1 S_m + g_2 S_{m-1} + r_2, where
//   g_1 = t_m iota_m, g_2 = t_{m-1} iota_{m-1} iota_m   (d psi_m / d S at those points),
//   r_1 = psi_{m-1} iota_m, r_2 = psi_{m-2} iota_{m-1} iota_m;
// so the entries of row ko of the inverse are Lambda*_{ko,k_j} = sigma g_j / D, and the
// effective intensity of bandwidth b keeps only the other lines' share of S at the band
// points: sigma (g_1 S_oth,m [+ g_2 S_oth,m-1] + r_b)/D, again a sum of non-negative terms.
// Missing points have g = 0 (and r_2 = r_1).
struct Side64 {
    double phi_iota, psi, dtau;
    double g[2], r[2], h[2], so[2];   // band weights, reduced psi, phi_l/chi and S_other at m, m-1
};

// Per-row history of the sweep for the band terms.
struct Row64 {
    double t, iota, psi_in, h, so;
};

template <int B, bool SCAT>
__device__ __forceinline__ Side64 sweep64(const SolveArgs &a, int l, double aq, double k1, double nu_o, int kstart,
                                          int kend, int step, const PairSmem64 &S, Pt64 &po) {
    // kstart: far end, kend: origin; step = +1 (backward half) or -1 (forward half)
    Pt64 p = point64<SCAT>(a, l, aq, k1, kstart, S);
    double chi_prev = fmax(p.chi, a.chi_min);
    double S_prev = p.eta / chi_prev;
    double h_prev = 0.0, so_prev = 0.0;
    if constexpr (B > 0) {
        h_prev = p.phil / chi_prev;
        so_prev = (p.eta - p.etal) / chi_prev;
    }
    const double I = planck_d(nu_o * (1.0 - S.v[kstart] / kC), a.T_cmb);
    double Phi = 0.0, iota = 0.0, psi = 0.0, dt_prev = 0.0;
    Row64 r1{0, 0, 0, 0, 0}, r2{0, 0, 0, 0, 0};
    int row = 0;
    for (int k = kstart + step;; k += step) {
        Pt64 q = point64<SCAT>(a, l, aq, k1, k, S);
        const double chi = fmax(q.chi, a.chi_min);
        const double Sk = q.eta / chi;
        const double dsk = S.ds[step > 0 ? k - 1 : k];
        const double dt = fmax(0.5 * (chi_prev + chi) * dsk, a.dtau_min);
        double t, psi_in;
        if (row == 0) {
            t = 0.5 * dt;
            psi_in = I;
            Phi = 0.5 * dt + 1.0;
            iota = 1.0 / (1.0 + dt * Phi);
            psi = (0.5 * dt * S_prev + I) * iota;
        } else {
            t = 0.5 * (dt_prev + dt);
            psi_in = psi;
            Phi = t + Phi * iota;
            iota = 1.0 / (1.0 + dt * Phi);
            psi = (t * S_prev + psi) * iota;
        }
        if constexpr (B > 0) {
            r2 = r1;
            r1 = Row64{t, iota, psi_in, h_prev, so_prev};
            h_prev = q.phil / chi;
            so_prev = (q.eta - q.etal) / chi;
        }
        row++;
        dt_prev = dt;
        chi_prev = chi;
        S_prev = Sk;
        if (k == kend) {
            q.chi = chi;
            po = q;
            break;
        }
    }
    Side64 s{Phi * iota, psi, dt_prev, {0.0, 0.0}, {psi, psi}, {0.0, 0.0}, {0.0, 0.0}};
    if constexpr (B > 0) {
        s.g[0] = r1.t * r1.iota;
        s.r[0] = r1.psi_in * r1.iota;
        s.h[0] = r1.h;
        s.so[0] = r1.so;
        s.r[1] = s.r[0];
        if (row >= 2) {
            s.g[1] = r2.t * r2.iota * r1.iota;
            s.r[1] = r2.psi_in * r2.iota * r1.iota;
            s.h[1] = r2.h;
            s.so[1] = r2.so;
        }
    }
    return s;
}

// NA accumulators per bin: sum u, L, Jeff, 1 - L, then Jeff of bandwidths 1..B.
template <int B, bool SCAT>
__global__ void k_feautrier64(SolveArgs a) {
    extern __shared__ double smem[];
    constexpr int NA = 4 + B;
    const int L = a.L, Q = a.Q, F = L * Q;
    const int kmax = a.kmax;
    // G groups of TG threads; with G > 1 each group is one warp and solves the pairs
    // p = g, g + G, ... of the point on its own staging buffers and partial sums (for
    // small F, so that a point keeps several warps busy); the partial sums are added in
    // group order at the end.
    const int G = a.groups;
    const int TG = blockDim.x / G;
    const int g = threadIdx.x / TG, t = threadIdx.x - g * TG;
    PairSmem64 S;
    S.ds = smem + (size_t)g * 4 * kmax;
    S.v = S.ds + kmax;
    S.ib = S.v + kmax;
    S.w = S.ib + kmax;
    double *acc_all = smem + (size_t)G * 4 * kmax;   // [G][F][NA]
    double *acc = acc_all + (size_t)g * NA * F;
    // band ALO: per pair, [G][F][2][B] coupling terms of the band points before the sum over bins
    double *mac = acc_all + (size_t)G * NA * F + (size_t)g * 2 * B * F;
    S.ca = reinterpret_cast<int32_t *>(acc_all + (size_t)G * (NA + 2 * B) * F) + (size_t)g * 2 * kmax;
    S.cb = S.ca + kmax;
    int64_t o = blockIdx.x;
    if (a.olist) {
        if ((int)blockIdx.x >= *a.ocount) return;
        o = a.olist[blockIdx.x];
    }
    for (int f = t; f < NA * F; f += TG) acc[f] = 0.0;
    const double bo = a.b[o];
    const double invP = 1.0 / a.P;
    for (int p = g; p < a.P; p += G) {
        const int rf = a.pf[p], rb = a.pb[p];
        const int64_t ofb = a.ray_off[o * a.R + rb], ofl = a.ray_off[o * a.R + rf];
        const int lb = (int)(a.ray_off[o * a.R + rb + 1] - ofb);
        const int lf = (int)(a.ray_off[o * a.R + rf + 1] - ofl);
        const int Kb = lb ? a.xcum[ofb + lb - 1] : 0;
        const int Kf = lf ? a.xcum[ofl + lf - 1] : 0;
        const int K = Kb + 1 + Kf;
        if (K > kmax) {
            if (t == 0) atomicOr(a.err, 2);
            continue;
        }
        if (G > 1) __syncwarp(); else __syncthreads();
        stage_half64(a, o, rb, Kb - 1, -1, S, t, TG);
        stage_half64(a, o, rf, Kb + 1, +1, S, t, TG);
        if (t == 0) {
            S.v[Kb] = 0.0;
            S.ib[Kb] = 1.0 / bo;
            S.w[Kb] = 0.0;
            S.ca[Kb] = (int32_t)o;
            S.cb[Kb] = (int32_t)o;
        }
        if (G > 1) __syncwarp(); else __syncthreads();
        for (int f = t; f < F; f += TG) {
            const int l = f / Q, q = f - l * Q;
            const double aq = a.roots[q] * bo;
            const double k1 = 1.0 + aq / kC;
            const double nu_o = a.lc[l].nu * k1;
            Side64 sb, sf;
            Pt64 po{0, 0, 0, 0, 0};
            double u, lam, uml, oml, jb[2] = {0.0, 0.0};
            if (K == 1) {
                const double I = planck_d(nu_o, a.T_cmb);
                u = I; lam = 0.0; uml = I; oml = 1.0;
                jb[0] = jb[1] = I;
                po = point64<SCAT>(a, l, aq, k1, Kb, S);
                po.chi = fmax(po.chi, a.chi_min);
                if (B > 0)
                    for (int j = 0; j < 2 * B; j++) mac[f * 2 * B + j] = 0.0;
            } else {
                if (Kb > 0) sb = sweep64<B, SCAT>(a, l, aq, k1, nu_o, 0, Kb, +1, S, po);
                if (Kf > 0) sf = sweep64<B, SCAT>(a, l, aq, k1, nu_o, K - 1, Kb, -1, S, po);
                if (Kb == 0 || Kf == 0) {
                    const double Io = planck_d(nu_o, a.T_cmb);
                    const Side64 empty{1.0, Io, 0.0, {0.0, 0.0}, {Io, Io}, {0.0, 0.0}, {0.0, 0.0}};
                    if (Kb == 0) sb = empty;
                    if (Kf == 0) sf = empty;
                }
                const double So = po.eta / po.chi;
                const double sig = 2.0 / (sb.dtau + sf.dtau);
                const double pi2 = sb.phi_iota + sf.phi_iota;
                const double D = 1.0 + sig * pi2;
                const double iD = 1.0 / D;
                u = (So + sig * (sb.psi + sf.psi)) * iD;
                lam = iD;
                uml = sig * (sb.psi + sf.psi) * iD;
                oml = sig * pi2 * iD;
                if constexpr (B > 0) {
                    const double rb1 = sb.g[0] * sb.so[0] + sb.r[0], rf1 = sf.g[0] * sf.so[0] + sf.r[0];
                    jb[0] = sig * (rb1 + rf1) * iD;
                    if constexpr (B > 1)
                        jb[1] = sig * (sb.g[0] * sb.so[0] + sb.g[1] * sb.so[1] + sb.r[1] +
                                       sf.g[0] * sf.so[0] + sf.g[1] * sf.so[1] + sf.r[1]) * iD;
                    const double sD = sig * iD;
                    for (int j = 0; j < B; j++) {
                        mac[f * 2 * B + j] = sD * sb.g[j] * sb.h[j];
                        mac[f * 2 * B + B + j] = sD * sf.g[j] * sf.h[j];
                    }
                }
            }
            const double ichi = 1.0 / po.chi;
            const double oth = lam * (po.eta - po.etal) * ichi;
            acc[NA * f + 0] += u;
            acc[NA * f + 1] += lam * po.chil * ichi;
            acc[NA * f + 2] += uml + oth;
            acc[NA * f + 3] += oml + lam * (po.chi - po.chil) * ichi;
            for (int j = 0; j < B; j++) acc[NA * f + 4 + j] += jb[j] + oth;
        }
        if constexpr (B > 0) {
            // coupling coefficients of this pair's band points: weighted sums over each
            // line's bins (fixed order), times chi_int,l(o)/P
            if (G > 1) __syncwarp(); else __syncthreads();
            for (int tk = t; tk < 2 * B * L; tk += TG) {
                const int l = tk / (2 * B), sj = tk - l * 2 * B;
                double s = 0.0;
                for (int q = 0; q < Q; q++) s += a.weights[q] * mac[(l * Q + q) * 2 * B + sj];
                const int side = sj / B, j = sj - side * B;
                const int r = side ? rf : rb;
                a.Mb[(((size_t)o * L + l) * a.R + r) * B + j] = s * invP * a.line[(o * L + l) * 2 + 1];
            }
        }
    }
    __syncthreads();
    for (int tt = threadIdx.x; tt < NA * L; tt += blockDim.x) {
        const int l = tt / NA, k = tt - l * NA;
        double s = 0.0;
        for (int q = 0; q < Q; q++) {
            double v = acc_all[NA * (l * Q + q) + k];
            for (int gg = 1; gg < G; gg++) v += acc_all[(size_t)gg * NA * F + NA * (l * Q + q) + k];
            s += a.weights[q] * v;
        }
        s *= invP;
        double *dst = k == 0 ? a.J : (k == 1 ? a.Lout : (k == 2 ? a.Jeff : (k == 3 ? a.Lc : a.Jeffb + (size_t)(k - 4) * a.n * L)));
        dst[o * L + l] = s;
    }
    if (a.Jnu)
        for (int f = threadIdx.x; f < F; f += blockDim.x) {
            double v = acc_all[NA * f];
            for (int gg = 1; gg < G; gg++) v += acc_all[(size_t)gg * NA * F + NA * f];
            a.Jnu[o * F + f] = v * invP;
        }
}

// ---------------------------------------------------------------- images
// Image along direction n (Sec. 3.5): each origin point o gives the intensity leaving the
// model along n on its ray pair, carried from the far end of the -n half to the far end
// of the n half with the first-order equation dI/dtau = S - I, the source linear in tau
// between points (Olson & Kunasz 1987):
//   I_{k+1} = e I_k + (alpha - e) S_k + (1 - alpha) S_{k+1},  e = exp(-dtau), alpha = (1 - e)/dtau,
// with the weights' Taylor series below dtau = 1e-3 (1 - alpha cancels there, and a
// floored opacity makes S as large as eta/chi_min).
// Channel c has rest-frame frequency nu_l (1 + u_c/c); at a point with rest-frame
// line-of-sight velocity w = n.v its comoving frequency is nu (1 - w/c). The staged pair
// holds each half's velocity relative to o along that half's own direction, so
// w = n.v_o - v on the -n half and n.v_o + v on the n half. All lines within reach of
// the channels (the host's list, which leaves out only lines whose profile underflows
// to zero everywhere) add to opacity and emissivity.
struct ImageArgs {
    SolveArgs s;              // ray store, widths, line data, floors, kmax, err
    int32_t rf, rb, n_ch, n_ov;
    const double *u;          // [n_ch]
    const Overlap *ov;        // [n_ov] lines within reach of the channels
    const double *vel;        // [n][3]
    const double *pos;        // [n][3]
    double n0, n1, n2;        // direction
    double e1[3], e2[3];      // sky-plane basis
    double nu_l;              // reference line frequency
    double *I;                // [n][n_ch]
    double *xy;               // [n][2]
    const float *dsf, *vparf, *bf, *linef;   // FP32 copies for the FP32 kernel
};

__device__ __forceinline__ double ls_step(double I, double d, double Sa, double Sb) {
    const double e = exp(-d);
    double wa, wb;
    if (d < 1e-3) {
        wb = d * (0.5 - d * (1.0 / 6.0 - d * (1.0 / 24.0 - d / 120.0)));
        wa = d * (0.5 - d * (1.0 / 3.0 - d * (1.0 / 8.0 - d / 30.0)));
    } else {
        const double alpha = -expm1(-d) / d;
        wb = 1.0 - alpha;
        wa = alpha - e;
    }
    return e * I + wa * Sa + wb * Sb;
}

__global__ void k_image64(ImageArgs a) {
    extern __shared__ double smem[];
    const SolveArgs &sa = a.s;
    const int kmax = sa.kmax;
    PairSmem64 S;
    S.ds = smem;
    S.v = S.ds + kmax;
    S.ib = S.v + kmax;
    S.w = S.ib + kmax;
    S.ca = reinterpret_cast<int32_t *>(S.w + kmax);
    S.cb = S.ca + kmax;
    const int64_t o = blockIdx.x;
    const double *xo = a.pos + 3 * o, *vo = a.vel + 3 * o;
    if (threadIdx.x == 0) {
        a.xy[2 * o] = xo[0] * a.e1[0] + xo[1] * a.e1[1] + xo[2] * a.e1[2];
        a.xy[2 * o + 1] = xo[0] * a.e2[0] + xo[1] * a.e2[1] + xo[2] * a.e2[2];
    }
    const double nvo = a.n0 * vo[0] + a.n1 * vo[1] + a.n2 * vo[2];
    const int64_t ofb = sa.ray_off[o * sa.R + a.rb], ofl = sa.ray_off[o * sa.R + a.rf];
    const int lb = (int)(sa.ray_off[o * sa.R + a.rb + 1] - ofb);
    const int lf = (int)(sa.ray_off[o * sa.R + a.rf + 1] - ofl);
    const int Kb = lb ? sa.xcum[ofb + lb - 1] : 0;
    const int Kf = lf ? sa.xcum[ofl + lf - 1] : 0;
    const int K = Kb + 1 + Kf;
    if (K > kmax) {
        if (threadIdx.x == 0) atomicOr(sa.err, 2);
        return;
    }
    stage_half64(sa, o, a.rb, Kb - 1, -1, S, threadIdx.x, blockDim.x);
    stage_half64(sa, o, a.rf, Kb + 1, +1, S, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        S.v[Kb] = 0.0;
        S.ib[Kb] = 1.0 / sa.b[o];
        S.w[Kb] = 0.0;
        S.ca[Kb] = (int32_t)o;
        S.cb[Kb] = (int32_t)o;
    }
    __syncthreads();
    constexpr double kCsp = kC / kSqrtPi;
    for (int c = threadIdx.x; c < a.n_ch; c += blockDim.x) {
        const double u = a.u[c];
        const double k1 = 1.0 + u / kC;
        double I = 0.0, chi_prev = 0.0, S_prev = 0.0;
        for (int k = 0; k < K; k++) {
            const double w = nvo + (k < Kb ? -S.v[k] : S.v[k]);
            const double ibk = S.ib[k], wt = S.w[k];
            const double *pa = sa.line + (int64_t)S.ca[k] * 2 * sa.L, *pb = sa.line + (int64_t)S.cb[k] * 2 * sa.L;
            const double base = u - w * k1;
            double eta = 0.0, chi = 0.0;
            for (int i = 0; i < a.n_ov; i++) {
                const Overlap ov = a.ov[i];
                const double x = (ov.dnl + ov.rat * base) * ibk;
                const double x2 = x * x;
                if (x2 > 746.0) continue;   // exp(-x^2) is zero in FP64
                const double phi = exp(-x2) * (ov.inv_nu2 * ibk) * kCsp;
                eta += ((1.0 - wt) * pa[2 * ov.l2] + wt * pb[2 * ov.l2]) * phi;
                chi += ((1.0 - wt) * pa[2 * ov.l2 + 1] + wt * pb[2 * ov.l2 + 1]) * phi;
            }
            chi = fmax(chi, sa.chi_min);
            const double Sk = eta / chi;
            if (k == 0) {
                I = planck_d(a.nu_l * k1 * (1.0 - w / kC), sa.T_cmb);
            } else {
                const double dt = fmax(0.5 * (chi_prev + chi) * S.ds[k - 1], sa.dtau_min);
                I = ls_step(I, dt, S_prev, Sk);
            }
            chi_prev = chi;
            S_prev = Sk;
        }
        a.I[o * a.n_ch + c] = I;
    }
}

// FP32 image of a mixed-precision context. The pair is staged once per point in shared
// memory in FP32 (from the FP32 ray store, widths and line data): path length,
// rest-frame line-of-sight velocity w, reciprocal width, and the interpolated (eta, chi)
// of the NOV lines within reach; then each thread carries one channel through the pair.
// The linear-source weights use their Taylor series below dtau = 0.05 (4 terms: relative
// error below 2e-8 there), where 1 - alpha would cancel in FP32; divisions are the fast
// approximate ones (2 ulp).
constexpr int kImgLines = 4;

struct ImgSmem32 {
    float *ds, *w, *ib, *lin;   // lin: [K][NOV][2] (eta, chi)
};

template <int NOV>
__device__ void stage_half_img32(const ImageArgs &a, int64_t o, int r, int base, int dir, float nvo, float sgn,
                                 const ImgSmem32 &S) {
    const SolveArgs &sa = a.s;
    const int64_t off = sa.ray_off[o * sa.R + r];
    const int len = (int)(sa.ray_off[o * sa.R + r + 1] - off);
    int l2[NOV];
#pragma unroll
    for (int i = 0; i < NOV; i++) l2[i] = a.ov[i].l2;
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int32_t c = sa.cells[off + e];
        const int32_t prev = e ? sa.cells[off + e - 1] : (int32_t)o;
        const int x0 = e ? sa.xcum[off + e - 1] : 0;
        const int ns = sa.xcum[off + e] - x0 - 1;
        const float pv = e ? a.vparf[off + e - 1] : 0.0f;
        const float ve = a.vparf[off + e];
        const float inv = 1.0f / (float)(ns + 1);
        const float dse = a.dsf[off + e] * inv;
        const float bp = a.bf[prev], bc = a.bf[c];
        const float *pa = a.linef + (int64_t)prev * 2 * sa.L, *pb = a.linef + (int64_t)c * 2 * sa.L;
        float la[NOV][2], lb[NOV][2];
#pragma unroll
        for (int i = 0; i < NOV; i++) {
            la[i][0] = pa[2 * l2[i]]; la[i][1] = pa[2 * l2[i] + 1];
            lb[i][0] = pb[2 * l2[i]]; lb[i][1] = pb[2 * l2[i] + 1];
        }
        for (int j = 1; j <= ns + 1; j++) {
            const float wt = (float)j * inv;
            const int idx = base + dir * (x0 + j - 1);
            S.ds[dir < 0 ? idx : idx - 1] = dse;
            S.w[idx] = nvo + sgn * ((1.0f - wt) * pv + wt * ve);
            S.ib[idx] = 1.0f / ((1.0f - wt) * bp + wt * bc);
#pragma unroll
            for (int i = 0; i < NOV; i++) {
                S.lin[(idx * NOV + i) * 2] = (1.0f - wt) * la[i][0] + wt * lb[i][0];
                S.lin[(idx * NOV + i) * 2 + 1] = (1.0f - wt) * la[i][1] + wt * lb[i][1];
            }
        }
    }
}

__device__ __forceinline__ float ls_step32(float I, float d, float Sa, float Sb) {
    const float e = __expf(-d);
    float wa, wb;
    if (d < 0.05f) {
        wb = d * (0.5f - d * (1.0f / 6.0f - d * (1.0f / 24.0f - d * (1.0f / 120.0f))));
        wa = d * (0.5f - d * (1.0f / 3.0f - d * (1.0f / 8.0f - d * (1.0f / 30.0f))));
    } else {
        const float alpha = __fdividef(1.0f - e, d);
        wb = 1.0f - alpha;
        wa = alpha - e;
    }
    return e * I + wa * Sa + wb * Sb;
}

// B_nu(T) in FP32, ordered so that no intermediate leaves the FP32 range.
__device__ __forceinline__ float planck_f(float nu, float T) {
    constexpr float k2h = (float)(2.0 * kH), kic = (float)(1.0 / kC), khk = (float)(kH / kKB);
    const float nc = nu * kic;
    return k2h * nc * nc * nu / expm1f(khk * nu / T);
}

template <int NOV>
__global__ void k_image32(ImageArgs a) {
    extern __shared__ float smf[];
    const SolveArgs &sa = a.s;
    const int kmax = sa.kmax;
    ImgSmem32 S;
    S.ds = smf;
    S.w = S.ds + kmax;
    S.ib = S.w + kmax;
    S.lin = S.ib + kmax;
    const int64_t o = blockIdx.x;
    const double *xo = a.pos + 3 * o, *vo = a.vel + 3 * o;
    if (threadIdx.x == 0) {
        a.xy[2 * o] = xo[0] * a.e1[0] + xo[1] * a.e1[1] + xo[2] * a.e1[2];
        a.xy[2 * o + 1] = xo[0] * a.e2[0] + xo[1] * a.e2[1] + xo[2] * a.e2[2];
    }
    const float nvo = (float)a.n0 * (float)vo[0] + (float)a.n1 * (float)vo[1] + (float)a.n2 * (float)vo[2];
    const int64_t ofb = sa.ray_off[o * sa.R + a.rb], ofl = sa.ray_off[o * sa.R + a.rf];
    const int lb = (int)(sa.ray_off[o * sa.R + a.rb + 1] - ofb);
    const int lf = (int)(sa.ray_off[o * sa.R + a.rf + 1] - ofl);
    const int Kb = lb ? sa.xcum[ofb + lb - 1] : 0;
    const int Kf = lf ? sa.xcum[ofl + lf - 1] : 0;
    const int K = Kb + 1 + Kf;
    if (K > kmax) {
        if (threadIdx.x == 0) atomicOr(sa.err, 2);
        return;
    }
    stage_half_img32<NOV>(a, o, a.rb, Kb - 1, -1, nvo, -1.0f, S);
    stage_half_img32<NOV>(a, o, a.rf, Kb + 1, +1, nvo, +1.0f, S);
    if (threadIdx.x == 0) {
        S.w[Kb] = nvo;
        S.ib[Kb] = 1.0f / a.bf[o];
        const float *pl = a.linef + o * 2 * sa.L;
#pragma unroll
        for (int i = 0; i < NOV; i++) {
            S.lin[(Kb * NOV + i) * 2] = pl[2 * a.ov[i].l2];
            S.lin[(Kb * NOV + i) * 2 + 1] = pl[2 * a.ov[i].l2 + 1];
        }
    }
    __syncthreads();
    constexpr float kCspf = (float)(kC / kSqrtPi);
    float dnl[NOV], rat[NOV], nrm[NOV];
#pragma unroll
    for (int i = 0; i < NOV; i++) {
        dnl[i] = (float)a.ov[i].dnl;
        rat[i] = (float)a.ov[i].rat;
        nrm[i] = (float)a.ov[i].inv_nu2 * kCspf;
    }
    const float chi_min = (float)sa.chi_min, dtau_min = (float)sa.dtau_min, T_cmb = (float)sa.T_cmb;
    const float nu_l = (float)a.nu_l, kic = (float)(1.0 / kC);
    for (int c = threadIdx.x; c < a.n_ch; c += blockDim.x) {
        const float u = (float)a.u[c];
        const float k1 = 1.0f + u * kic;
        float I = 0.0f, chi_prev = 0.0f, S_prev = 0.0f;
        for (int k = 0; k < K; k++) {
            const float w = S.w[k], ibk = S.ib[k];
            const float base = u - w * k1;
            float eta = 0.0f, chi = 0.0f;
#pragma unroll
            for (int i = 0; i < NOV; i++) {
                const float x = (dnl[i] + rat[i] * base) * ibk;
                const float phi = __expf(-x * x) * (nrm[i] * ibk);
                eta += S.lin[(k * NOV + i) * 2] * phi;
                chi += S.lin[(k * NOV + i) * 2 + 1] * phi;
            }
            chi = fmaxf(chi, chi_min);
            const float Sk = __fdividef(eta, chi);
            if (k == 0) {
                I = planck_f(nu_l * k1 * (1.0f - w * kic), T_cmb);
            } else {
                const float dt = fmaxf(0.5f * (chi_prev + chi) * S.ds[k - 1], dtau_min);
                I = ls_step32(I, dt, S_prev, Sk);
            }
            chi_prev = chi;
            S_prev = Sk;
        }
        a.I[o * a.n_ch + c] = (double)I;
    }
}

}  // namespace

namespace {
// Largest |a_new - a_old| / a_new over m values into *word (as the bits of a double, which
// order like the values for non-negative doubles); NaN counts as infinity.
__global__ void k_vec_max_rel_change(int64_t m, const double *a_new, const double *a_old, unsigned long long *word) {
    double mx = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        double d = fabs(a_new[i] - a_old[i]) / a_new[i];
        if (!(d <= INFINITY)) d = INFINITY;
        mx = fmax(mx, d);
    }
    unsigned long long bits = __double_as_longlong(mx);
    for (int d = 16; d; d >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, bits, d);
        bits = o > bits ? o : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(word, bits);
}
}  // namespace

int mg_launch_max_rel_change(mg_ctx *ctx, int64_t m, const double *a_new, const double *a_old,
                             unsigned long long *word) {
    MG_CUDA(cudaMemsetAsync(word, 0, sizeof(unsigned long long), ctx->stream));
    k_vec_max_rel_change<<<4 * 152, 256, 0, ctx->stream>>>(m, a_new, a_old, word);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_line_data(mg_ctx *ctx) {
    if (ctx->opt.precision == MG_MIXED) return mg_launch_line_data_mixed(ctx);
    const int64_t m = ctx->n * ctx->n_lines;
    MgTimed t(ctx, "line_data");
    k_line_data<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->n, ctx->n_lines, ctx->n_lev, ctx->d_pops, ctx->d_lines, ctx->d_line, nullptr, ctx->d_scal + 4);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_feautrier_mixed(mg_ctx *ctx);

// Cells whose largest diagonal ALO weight over the lines is >= lmin go to the list.
__global__ void k_mark_thick(int64_t n, int L, const double *Lw, double lmin, int32_t *list, int32_t *count) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double mx = 0.0;
    for (int l = 0; l < L; l++) mx = fmax(mx, Lw[c * L + l]);
    if (mx >= lmin) list[atomicAdd(count, 1)] = (int32_t)c;
}

static int launch_fp64(mg_ctx *ctx, const int32_t *olist, const int32_t *ocount, unsigned grid);

int mg_launch_feautrier_fp64_list(mg_ctx *ctx, const int32_t *olist, const int32_t *ocount) {
    return launch_fp64(ctx, olist, ocount, (unsigned)ctx->n);
}

int mg_launch_feautrier(mg_ctx *ctx) {
    if (ctx->opt.precision == MG_MIXED) {
        int rc = mg_launch_feautrier_mixed(ctx);
        if (rc || !(ctx->opt.tau_fp64 > 0.0)) return rc;
        // FP64 promotion of optically thick cells: list them, then solve them again in FP64
        if (!ctx->d_promo && (rc = mg_alloc(ctx, &ctx->d_promo, ctx->n + 1))) return rc;
        MG_CUDA(cudaMemsetAsync(ctx->d_promo + ctx->n, 0, sizeof(int32_t), ctx->stream));
        k_mark_thick<<<(unsigned)((ctx->n + 255) / 256), 256, 0, ctx->stream>>>(
            ctx->n, ctx->n_lines, ctx->d_L, 1.0 - 1.0 / ctx->opt.tau_fp64, ctx->d_promo, ctx->d_promo + ctx->n);
        MG_CUDA(cudaGetLastError());
        return launch_fp64(ctx, ctx->d_promo, ctx->d_promo + ctx->n, (unsigned)ctx->n);
    }
    return launch_fp64(ctx, nullptr, nullptr, (unsigned)ctx->n);
}

static int launch_fp64(mg_ctx *ctx, const int32_t *olist, const int32_t *ocount, unsigned grid) {
    SolveArgs a{};
    a.n = ctx->n; a.R = ctx->R; a.P = ctx->P; a.L = ctx->n_lines; a.Q = ctx->Q;
    a.pf = ctx->d_pf; a.pb = ctx->d_pb; a.ray_off = ctx->d_ray_off; a.cells = ctx->d_cells; a.xcum = ctx->d_xcum;
    a.ds = ctx->d_ds; a.vpar = ctx->d_vpar; a.b = ctx->d_b; a.line = ctx->d_line; a.lc = ctx->d_lines;
    a.roots = ctx->d_roots; a.weights = ctx->d_weights; a.ovl_off = ctx->d_ovl_off; a.ovl = ctx->d_ovl;
    a.chi_min = ctx->opt.chi_min; a.dtau_min = ctx->opt.dtau_min; a.T_cmb = ctx->opt.T_cmb;
    a.J = ctx->d_J; a.Lout = ctx->d_L; a.Jeff = ctx->d_Jeff; a.Lc = ctx->d_Lc;
    a.Jnu = ctx->opt.spectrum ? ctx->d_Jnu : nullptr;
    a.kmax = (int32_t)ctx->max_pair_len;
    a.err = ctx->d_err;
    a.olist = olist;
    a.ocount = ocount;
    const int B = olist ? 0 : ctx->band_cur;   // the band ALO is built for FP64 contexts
    a.Jeffb = ctx->d_Jeffb;
    a.Mb = ctx->d_Mb;
    const int F = a.L * a.Q;
    auto smem_for = [&](int G) {
        return (size_t)G * (sizeof(double) * ((size_t)a.kmax * 4 + (4 + 3 * (size_t)B) * F) +
                            sizeof(int32_t) * 2 * (size_t)a.kmax);
    };
    size_t smem = smem_for(1);
    if (smem > 227 * 1024)
        return mg_fail(ctx, MG_ERR_CAPACITY, "FP64 formal solve: longest ray pair does not fit in shared memory");
    // up to 8 warps per point solve different ray pairs when one warp covers all bins,
    // as many as two CTAs per SM leave room for, balanced over the pairs
    a.groups = 1;
    if (F <= 32) {
        int gmax = 1;
        while (gmax < 8 && gmax < a.P && smem_for(gmax + 1) <= 113 * 1024) gmax++;
        const int rounds = (a.P + gmax - 1) / gmax;
        a.groups = (a.P + rounds - 1) / rounds;
    }
    smem = smem_for(a.groups);
    const bool sca = !olist && ctx->sca_on;
    void (*kern)(SolveArgs) = sca ? (B == 0 ? k_feautrier64<0, true> : (B == 1 ? k_feautrier64<1, true> : k_feautrier64<2, true>))
                                  : (B == 0 ? k_feautrier64<0, false> : (B == 1 ? k_feautrier64<1, false> : k_feautrier64<2, false>));
    if (sca) {
        a.chi_sca = ctx->d_chisca;
        a.Jsca = ctx->d_Jsca;
        a.Jnu = ctx->d_Jsca_new;
    }
    MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int threads = a.groups > 1 ? 32 * a.groups : ((F + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    if (!olist) MG_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
    {
        MgTimed t(ctx, olist ? "feautrier_fp64_promoted" : "feautrier_fp64");
        kern<<<grid, threads, smem, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

// FP64 line data (and its plain FP32 copy when linef is given) from the current
// populations, for the images in either precision.
int mg_launch_line_data64(mg_ctx *ctx, float *linef, unsigned long long *neg) {
    const int64_t m = ctx->n * ctx->n_lines;
    k_line_data<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->n, ctx->n_lines, ctx->n_lev, ctx->d_pops, ctx->d_lines, ctx->d_line, linef, neg);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

int mg_launch_image(mg_ctx *ctx, int ray, int line, int n_ch, const double *d_u, const Overlap *d_ov, int n_ov,
                    double *d_I, double *d_xy) {
    ImageArgs a{};
    SolveArgs &s = a.s;
    s.n = ctx->n; s.R = ctx->R; s.P = ctx->P; s.L = ctx->n_lines; s.Q = ctx->Q;
    s.ray_off = ctx->d_ray_off; s.cells = ctx->d_cells; s.xcum = ctx->d_xcum;
    s.ds = ctx->d_ds; s.vpar = ctx->d_vpar; s.b = ctx->d_b; s.line = ctx->d_line; s.lc = ctx->d_lines;
    s.chi_min = ctx->opt.chi_min; s.dtau_min = ctx->opt.dtau_min; s.T_cmb = ctx->opt.T_cmb;
    s.kmax = (int32_t)ctx->max_pair_len;
    s.err = ctx->d_err;
    a.rf = ray;
    a.rb = ctx->h_anti[ray];
    a.n_ch = n_ch;
    a.n_ov = n_ov;
    a.u = d_u;
    a.ov = d_ov;
    a.vel = ctx->d_vel;
    a.pos = ctx->d_pos;
    const double *n = &ctx->h_dirs[3 * (size_t)ray];
    a.n0 = n[0]; a.n1 = n[1]; a.n2 = n[2];
    // e1 = (z x n)/|z x n| (x in place of z when |n_z| >= 0.9), e2 = n x e1
    double ax[3] = {0.0, 0.0, 1.0};
    if (std::fabs(n[2]) >= 0.9) { ax[0] = 1.0; ax[2] = 0.0; }
    double e1[3] = {ax[1] * n[2] - ax[2] * n[1], ax[2] * n[0] - ax[0] * n[2], ax[0] * n[1] - ax[1] * n[0]};
    const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double &v : e1) v /= l1;
    a.e1[0] = e1[0]; a.e1[1] = e1[1]; a.e1[2] = e1[2];
    a.e2[0] = n[1] * e1[2] - n[2] * e1[1];
    a.e2[1] = n[2] * e1[0] - n[0] * e1[2];
    a.e2[2] = n[0] * e1[1] - n[1] * e1[0];
    a.nu_l = ctx->h_lines[line].nu;
    a.I = d_I;
    a.xy = d_xy;
    int threads = ((n_ch + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    MG_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
    // FP32 in a mixed-precision context when the lines within reach fit the staging
    a.dsf = ctx->d_dsf; a.vparf = ctx->d_vparf; a.bf = ctx->d_bf; a.linef = ctx->d_imglf;
    const size_t smem32 = sizeof(float) * (size_t)s.kmax * (3 + 2 * (size_t)n_ov);
    if (ctx->opt.precision == MG_MIXED && n_ov <= kImgLines && smem32 <= 227 * 1024 && a.linef) {
        void (*kern)(ImageArgs) = n_ov == 1 ? k_image32<1> : n_ov == 2 ? k_image32<2> : n_ov == 3 ? k_image32<3>
                                                                                                  : k_image32<4>;
        MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
        MgTimed t(ctx, "image_fp32");
        kern<<<(unsigned)ctx->n, threads, smem32, ctx->stream>>>(a);
    } else {
        const size_t smem = sizeof(double) * (size_t)s.kmax * 4 + sizeof(int32_t) * 2 * (size_t)s.kmax;
        if (smem > 227 * 1024)
            return mg_fail(ctx, MG_ERR_CAPACITY, "mg_image: longest ray pair does not fit in shared memory");
        MG_CUDA(cudaFuncSetAttribute(k_image64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MgTimed t(ctx, "image_fp64");
        k_image64<<<(unsigned)ctx->n, threads, smem, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}
