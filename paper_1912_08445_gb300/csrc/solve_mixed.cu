// K3 in mixed precision: the Feautrier formal solve of Sec. 3.3-3.4 in FP32 (the
// statistical equilibrium that follows stays in FP64). Intensities are carried in units
// of I0 = 1e-20 W m^-2 Hz^-1 sr^-1 and the float line data are scaled (chi x 1e5,
// eta x 1e25) so that no FP32 quantity underflows. The line opacity of bin a_q at a point
// is chi_l = X 2^(-x'^2), with X = chi_int c / (nu_l b sqrt(pi)) and the profile
// argument x' in units of sqrt(log2 e) Doppler widths; for a line that overlaps no other
// line the source function S = eta_int/chi_int is frequency independent.
//
// Two kernels:
// - k_feautrier_warp (the common case: lines that do not overlap) gives each warp one
//   origin and a group of G lines, with the bins of those lines across its lanes (NB
//   per lane), and sweeps every ray pair through a per-warp ring of staged points; the
//   persistent k_feautrier_batch runs the same work item over a queue of models.
// - k_feautrier_mixed (lines that overlap, so that a bin sums several lines) gives each
//   origin a CTA and stages every ray pair whole in shared memory.
//
// Per point and bin the sweep costs one ex2 and one rcp (MUFU) and a handful of FMA-
// and ALU-pipe ops, in the rescaled Rybicki-Hummer recursion described with the FP64
// kernel:
//   dtau = max((chi_prev + chi) ds/2, dtau_min),  t = (dtau_prev + dtau)/2,
//   Phi = t + Phi iota,  iota = 1/(1 + dtau Phi),  psi = (t S + psi) iota.
#include <cmath>
#include <cstring>
#include <type_traits>
#include "common.cuh"

using namespace mg;

namespace {

constexpr float kSqrtLog2e = 1.2011224087864498f;
constexpr float kSqrt2 = 1.4142135623730951f;
constexpr float kInvSqrt8 = 0.35355339059327373f;   // 1/(2 sqrt 2)
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpf(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void k_line_data_f32(int64_t n, int L, int nlev, const double *__restrict__ pops,
                                const LineConst *__restrict__ lc, double *__restrict__ line,
                                float *__restrict__ linef, unsigned long long *neg) {
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
    // (eta, chi) times the profile normalisation c / (nu_l sqrt(pi)): the line opacity of a
    // bin is then chi' 2^(-x'^2) / b, and S = eta'/chi' keeps the scale kEtaScale/kChiScale
    const double kl = kC / (k.nu * kSqrtPi);
    linef[2 * t] = (float)(eta * (kEtaScale / kChiScale) * kl);
    linef[2 * t + 1] = (float)(chi * kl);
}

struct MixArgs {
    int64_t n;
    int32_t R, P, L, Q;
    const int32_t *pf, *pb;
    const int64_t *ray_off;
    const int32_t *cells, *xcum;
    const float *ds, *vpar, *b;
    const float *line;           // [n][L][2] (eta, chi) times c/(nu_l sqrt(pi)), eta also times kEtaScale/kChiScale
    const float *nu_ghz;         // [L]
    const double *roots, *weights;
    const int32_t *ovl_off;
    const Overlap *ovl;
    float chi_min, dtau_min, inv_chi_min;
    float q_nofloor;             // q' = chi_min ds/(2 sqrt 2) from which 2 q' >= dtau_min in FP32
    float qscale;                // chi_min/(2 sqrt 2): q' of an interval per unit length
    float planck_a, planck_b;    // B'(nu) = a nu_G^3 / expm1(b nu_G): a = 2h 1e27/c^2/I0, b = h 1e9/(k T_cmb)
    double *J, *Lout, *Jeff, *Lc, *Jnu;
    int32_t kmax;
    int32_t overlap;             // some line overlaps another
    int32_t *err;
    unsigned long long *work;    // optional: point-bin updates the warp kernel executed
};

__device__ __forceinline__ float planck_f(const MixArgs &a, float nu_g) {
    return a.planck_a * nu_g * nu_g * nu_g / expm1f(a.planck_b * nu_g);
}

// CTA kernel (overlapping lines). Stages half-ray (o, r) in FP32, point x of the half at
// pair index base + dir x:
//   pt[k]    = (ds_k / 2, v_k, sqrt(log2 e)/b_k, 0)
//   ln[k][l] = (X_l, S_l) of every line l.
__device__ void stage_half32(const MixArgs &a, int64_t o, int r, int base, int dir, float4 *pt, float2 *ln) {
    const int L = a.L;
    const int64_t off = a.ray_off[o * a.R + r];
    const int len = (int)(a.ray_off[o * a.R + r + 1] - off);
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int64_t c = a.cells[off + e];
        const int64_t prev = e ? a.cells[off + e - 1] : o;
        const int x0 = e ? a.xcum[off + e - 1] : 0;
        const int ns = a.xcum[off + e] - x0 - 1;
        const float pv = e ? a.vpar[off + e - 1] : 0.0f;
        const float ve = a.vpar[off + e];
        const float hds = 0.5f * a.ds[off + e] / (float)(ns + 1);
        const float bp = a.b[prev], bc = a.b[c];
        const float2 *lp = reinterpret_cast<const float2 *>(a.line) + prev * L;
        const float2 *lq = reinterpret_cast<const float2 *>(a.line) + c * L;
        for (int j = 1; j <= ns + 1; j++) {
            const float w = (float)j / (float)(ns + 1);
            const int idx = base + dir * (x0 + j - 1);
            const float bb = (1.0f - w) * bp + w * bc;
            const float ib = 1.0f / bb;
            // the path length is stored with the point farther from the origin
            pt[idx] = make_float4(hds, (1.0f - w) * pv + w * ve, kSqrtLog2e * ib, 0.0f);
            for (int l = 0; l < L; l++) {
                const float2 p0 = lp[l], p1 = lq[l];
                const float et = (1.0f - w) * p0.x + w * p1.x;
                const float ch = (1.0f - w) * p0.y + w * p1.y;
                const float X = ch * ib;
                const float S = ch > 0.0f ? et / ch : 0.0f;
                ln[(size_t)idx * L + l] = make_float2(X, S);
            }
        }
    }
}

struct Side32 {
    float phi_iota, psi, dtau;
};

// Opacity and emissivity at point k for bin (l, aq); fast path: line l alone.
template <bool OVL>
__device__ __forceinline__ void point32(const MixArgs &a, int l, float aq, float A1, int k, const float4 *pt,
                                        const float2 *ln, float &chi, float &S, float &chil, float &etal) {
    const float4 p = pt[k];
    if (!OVL) {
        const float2 d = ln[(size_t)k * a.L + l];
        const float x = fmaf(-p.y, A1, aq) * p.z;
        const float e = ex2f(-x * x);
        chil = d.x * e;
        etal = chil * d.y;
        if (chil >= a.chi_min) {
            chi = chil;
            S = d.y;
        } else {   // opacity floor: S = eta / chi_min
            chi = a.chi_min;
            S = etal * a.inv_chi_min;
        }
        return;
    }
    // general case: sum over the lines that can reach this bin
    float ch = 0.f, et = 0.f;
    const int o0 = a.ovl_off[l], o1 = a.ovl_off[l + 1];
    const float base = fmaf(-p.y, A1, aq);
    for (int i = o0; i < o1; i++) {
        const Overlap ov = a.ovl[i];
        const float2 d = ln[(size_t)k * a.L + ov.l2];
        const float x = ((float)ov.dnl + (float)ov.rat * base) * p.z;
        const float c2 = d.x * ex2f(-x * x);
        ch += c2;
        et += c2 * d.y;
        if (i == o0) { chil = c2; etal = c2 * d.y; }
    }
    chi = fmaxf(ch, a.chi_min);
    S = et / chi;
}

template <bool OVL>
__device__ __forceinline__ Side32 sweep32(const MixArgs &a, int l, float aq, float A1, float nu_og, int kstart,
                                          int kend, int step, const float4 *pt, const float2 *ln, float &chi_o,
                                          float &S_o, float &chil_o, float &etal_o) {
    float chi_p, S_p, cl, el;
    point32<OVL>(a, l, aq, A1, kstart, pt, ln, chi_p, S_p, cl, el);
    const float I = planck_f(a, nu_og * (1.0f - pt[kstart].y * (float)(1.0 / kC)));
    float Phi, iota, psi, dt_p;
    // boundary row (first interval)
    {
        const int k = kstart + step;
        float chi, S;
        point32<OVL>(a, l, aq, A1, k, pt, ln, chi, S, cl, el);
        const float hds = pt[kstart].x;   // interval (kstart, k): stored with the farther point
        const float dt = fmaxf((chi_p + chi) * hds, a.dtau_min);
        Phi = fmaf(0.5f, dt, 1.0f);
        iota = rcpf(fmaf(dt, Phi, 1.0f));
        psi = fmaf(0.5f * dt, S_p, I) * iota;
        dt_p = dt;
        chi_p = chi;
        S_p = S;
        if (k == kend) {
            chi_o = chi; S_o = S; chil_o = cl; etal_o = el;
            return Side32{Phi * iota, psi, dt_p};
        }
    }
    for (int k = kstart + 2 * step;; k += step) {
        float chi, S;
        point32<OVL>(a, l, aq, A1, k, pt, ln, chi, S, cl, el);
        const float hds = pt[k - step].x;
        const float dt = fmaxf((chi_p + chi) * hds, a.dtau_min);
        const float t = 0.5f * (dt_p + dt);
        Phi = fmaf(Phi, iota, t);
        iota = rcpf(fmaf(dt, Phi, 1.0f));
        psi = fmaf(t, S_p, psi) * iota;
        dt_p = dt;
        chi_p = chi;
        S_p = S;
        if (k == kend) {
            chi_o = chi; S_o = S; chil_o = cl; etal_o = el;
            break;
        }
    }
    return Side32{Phi * iota, psi, dt_p};
}

// Shared memory of the CTA kernel: pt [kmax] float4, ln [kmax][L] float2, then acc
// [L][Q] float4 at the next 16-byte boundary.
__host__ __device__ constexpr size_t mixed_acc_offset(int kmax, int L) {
    return (16 * (size_t)kmax + 8 * (size_t)kmax * L + 15) & ~(size_t)15;
}
static_assert(mixed_acc_offset(3, 3) % 16 == 0 && mixed_acc_offset(3, 3) >= 16 * 3 + 8 * 9, "acc alignment");
static_assert(mixed_acc_offset(4, 2) == 16 * 4 + 8 * 8, "no padding when kmax * L is even");

template <bool OVL>
__global__ void __launch_bounds__(256) k_feautrier_mixed(MixArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.L, Q = a.Q;
    const int kmax = a.kmax;
    float4 *pt = reinterpret_cast<float4 *>(smem_raw);
    float2 *ln = reinterpret_cast<float2 *>(pt + kmax);
    // [L*Q]: (sum u, L, Jeff, 1-L); starts on a 16-byte boundary (kmax * L may be odd)
    float4 *acc = reinterpret_cast<float4 *>(smem_raw + mixed_acc_offset(kmax, L));
    const int64_t o = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int f = threadIdx.x; f < L * Q; f += blockDim.x) acc[f] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float bo = a.b[o];
    const float2 *lo = reinterpret_cast<const float2 *>(a.line) + o * L;
    for (int p = 0; p < a.P; p++) {
        const int rf = a.pf[p], rb = a.pb[p];
        const int64_t ofb = a.ray_off[o * a.R + rb], ofl = a.ray_off[o * a.R + rf];
        const int lb = (int)(a.ray_off[o * a.R + rb + 1] - ofb);
        const int lf = (int)(a.ray_off[o * a.R + rf + 1] - ofl);
        const int Kb = lb ? a.xcum[ofb + lb - 1] : 0;
        const int Kf = lf ? a.xcum[ofl + lf - 1] : 0;
        const int K = Kb + 1 + Kf;
        if (K > kmax) {
            if (threadIdx.x == 0) atomicOr(a.err, 2);
            continue;
        }
        __syncthreads();
        stage_half32(a, o, rb, Kb - 1, -1, pt, ln);
        stage_half32(a, o, rf, Kb + 1, +1, pt, ln);
        if (threadIdx.x == 0) pt[Kb] = make_float4(0.f, 0.f, kSqrtLog2e / bo, 0.f);
        for (int l = threadIdx.x; l < L; l += blockDim.x) {
            const float2 d = lo[l];
            const float X = d.y / bo;
            ln[(size_t)Kb * L + l] = make_float2(X, d.y > 0.f ? d.x / d.y : 0.f);
        }
        __syncthreads();
        for (int l = warp; l < L; l += nwarps) {
            const float nu_g = a.nu_ghz[l];
            for (int q = lane; q < Q; q += 32) {
                const float aq = (float)(a.roots[q] * a.b[o]);
                const float A1 = 1.0f + aq * (float)(1.0 / kC);
                const float nu_og = nu_g * A1;
                float u, lam, uml, oml, chi_o = 0.f, S_o = 0.f, chil = 0.f, etal = 0.f;
                if (K == 1) {
                    const float I = planck_f(a, nu_og);
                    point32<OVL>(a, l, aq, A1, Kb, pt, ln, chi_o, S_o, chil, etal);
                    u = I; lam = 0.f; uml = I; oml = 1.f;
                } else {
                    Side32 sb{1.f, 0.f, 0.f}, sf{1.f, 0.f, 0.f};
                    if (Kb > 0) sb = sweep32<OVL>(a, l, aq, A1, nu_og, 0, Kb, +1, pt, ln, chi_o, S_o, chil, etal);
                    if (Kf > 0) sf = sweep32<OVL>(a, l, aq, A1, nu_og, K - 1, Kb, -1, pt, ln, chi_o, S_o, chil, etal);
                    if (Kb == 0 || Kf == 0) {
                        const float Io = planck_f(a, nu_og);
                        if (Kb == 0) sb.psi = Io;
                        if (Kf == 0) sf.psi = Io;
                    }
                    const float sig = 2.0f / (sb.dtau + sf.dtau);
                    const float pi2 = sb.phi_iota + sf.phi_iota;
                    const float iD = 1.0f / fmaf(sig, pi2, 1.0f);
                    const float ps = sig * (sb.psi + sf.psi);
                    u = (S_o + ps) * iD;
                    lam = iD;
                    uml = ps * iD;
                    oml = sig * pi2 * iD;
                }
                const float ichi = 1.0f / chi_o;
                const float eta_o = S_o * chi_o;
                float4 r = acc[l * Q + q];
                r.x += u;
                r.y += lam * chil * ichi;
                r.z += uml + lam * (eta_o - etal) * ichi;
                r.w += oml + lam * (chi_o - chil) * ichi;
                acc[l * Q + q] = r;
            }
        }
    }
    __syncthreads();
    // per-line weighted sums over bins, fixed order, in FP64
    const double invP = 1.0 / a.P;
    for (int t = threadIdx.x; t < 4 * L; t += blockDim.x) {
        const int l = t >> 2, k = t & 3;
        double s = 0.0;
        for (int q = 0; q < Q; q++) {
            const float4 r = acc[l * Q + q];
            const float v = k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
            s += a.weights[q] * (double)v;
        }
        s *= invP;
        if (k == 0 || k == 2) s *= (double)kI0;
        double *dst = k == 0 ? a.J : (k == 1 ? a.Lout : (k == 2 ? a.Jeff : a.Lc));
        dst[o * L + l] = s;
    }
    if (a.Jnu)
        for (int f = threadIdx.x; f < L * Q; f += blockDim.x) a.Jnu[o * L * Q + f] = (double)acc[f].x * invP * (double)kI0;
}


// ---------------------------------------------------------------------------------
// Warp-per-(origin, line group) variant for models whose lines do not overlap (the
// common case). A warp serves G lines (G lane groups of 32/G lanes) and every lane NB
// bins of its line, so each shared-memory read and loop step is shared by NB updates.
// The warp loops over all ray pairs of its origin and stages the expanded points through
// a private ring of kRing points (one point per lane per refill): no CTA barrier is ever
// needed, and the pair sums are kept per lane in a fixed order. The boundary row is the
// interior update started from the virtual state (Phi iota = 1, psi = I, dtau = 0).
// The opacity floor: chi = max(chi_l, chi_min) and S_eff = S min(chi_l/chi_min, 1),
// which is eta/chi with chi floored. The warp kernel carries opacities in units of
// chi_min (and the interval factor q times chi_min, so that dtau is unchanged): the floor
// is then max(chi', 1) and the source's min(chi', 1), with no multiplication by
// 1/chi_min per bin.
//
// The ray elements behind the ring come from an element window in shared memory (one
// element per lane). A window serves refills until its points are used up; meanwhile
// the next window is filled asynchronously (cp.async): its records (xcum, cell, v, ds)
// are issued on the first refill from the current window, and the gathers through the
// cell index (b and the line data) half-way through that refill's sweep, so a window is
// normally complete when it is needed. The last window of a half-ray prefetches the
// first window of the next half-ray.
constexpr int kRing = 32;
constexpr int kWarps2 = 4;   // warps per block of most launch variants
constexpr int kWin = 32;   // elements top, top-1, ..., top-31 of a half-ray

// Element window of one warp, double-buffered: one slot per lane. Element e of the
// half-ray sits at slot top - e; element -1 (reached when top < 31) is the origin itself:
// xcum 0, cell o, v 0. Slots 0 .. 30 own the points of a refill; slot 31 only serves as
// the predecessor (towards the origin) of slot 30.
template <int G>
struct ElemWin {
    int32_t x1[2][kWin];      // xcum[e]: the element's expanded points are xcum[e-1] .. xcum[e]-1
    int32_t cell[2][kWin];
    float ds[2][kWin];
    float2 vb[2][kWin];        // (line-of-sight velocity, width b) of the element's cell
    float2 ln[2][G][kWin];    // scaled (eta, chi) of the warp's lines at the element's cell
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issues the copies of the records of elements top .. top-31 of the half-ray at `off`
// into buffer bf (lane i: slot i).
template <int G>
__device__ __forceinline__ void win_records(const MixArgs &a, int64_t off, int top, int32_t o, ElemWin<G> &w,
                                            int bf) {
    const int i = threadIdx.x & 31;
    const int e = top - i;
    if (e >= 0) {
        const int64_t k = off + e;
        cp_async4(&w.x1[bf][i], a.xcum + k);
        cp_async4(&w.cell[bf][i], a.cells + k);
        cp_async4(&w.vb[bf][i].x, a.vpar + k);
        cp_async4(&w.ds[bf][i], a.ds + k);
    } else {
        w.x1[bf][i] = 0;
        w.cell[bf][i] = o;
        w.vb[bf][i].x = 0.0f;
        w.ds[bf][i] = 0.0f;
    }
    cp_async_commit();
}

// Issues the gathers through the cell index of buffer bf; the records must have landed
// (each lane reads only the slots it copied itself).
template <int G>
__device__ __forceinline__ void win_gathers(const MixArgs &a, int l0, ElemWin<G> &w, int bf) {
    const int i = threadIdx.x & 31;
    const int64_t c = w.cell[bf][i];
    cp_async4(&w.vb[bf][i].y, a.b + c);
    const float2 *lc = reinterpret_cast<const float2 *>(a.line) + c * a.L;
#pragma unroll
    for (int k = 0; k < G; k++) cp_async8(&w.ln[bf][k][i], lc + (l0 + k < a.L ? l0 + k : a.L - 1));
    cp_async_commit();
}

// Scalars of the sweep, held in registers (not re-read from the argument block).
struct SweepK {
    float dtau_min, planck_a, planck_b;
};

// B_nu / I0 at nu_g GHz; e^x - 1 from one ex2 (x = h nu / k T_cmb is O(1) at line
// frequencies, so the subtraction costs no precision there).
__device__ __forceinline__ float planck_k(const SweepK &k, float nu_g) {
    return k.planck_a * nu_g * nu_g * nu_g * rcpf(ex2f(k.planck_b * kLog2e * nu_g) - 1.0f);
}

// One staged point of the ring. The per-point scalars are stored twice so that a bin
// pair reads them as the operand pairs of packed FP32x2 arithmetic:
//   a = (g_z, g_z, -g_y, -g_y) with g_y = sqrt(log2 e) v/b and g_z = sqrt(log2 e)(1 - v/c)/b,
//       so that the profile argument of bin a_q is x' = a_q g_z - g_y;
//   b = (q', q', far, 0) with q' = chi_min ds/(2 sqrt 2) to the next point towards the
//       origin (the half-width interval factor that yields delta = dtau/sqrt 2 from
//       opacities in units of chi_min).
// The line data of a point are (X', X', S, S) per line, X' = X/chi_min: the line opacity
// in units of chi_min is chi' = X' 2^(-x'^2), the floored opacity max(chi', 1), and the
// floored source S_eff = S min(chi', 1), which is eta/chi with chi = max(chi_l, chi_min)
// (exactly S where the line is not floored; finite for any finite S).
struct RingPt {
    float4 a, b;
};

// Expanded point x of the element in window slot i (sub-point (x - x0 + 1)/(ns + 1) of the
// interval from the element's predecessor towards the origin to its own cell).
// A point is "far" for the warp when every bin of the warp lies so far in the wings of
// every line of its group that the opacity is floored there: X 2^(-x'^2) < chi_min with
// x' = a_q g_z - g_y over the warp's range of a_q (monotonic in a_q, so the smallest
// |x'| is at an end of the range or zero). The divisions here use the approximate
// reciprocal (the path computes in FP32).
template <int G>
__device__ __forceinline__ void stage_ring_point(const MixArgs &a, const ElemWin<G> &w, int bf, int i, int l0, int x,
                                                 RingPt &pt, float4 *ln, float aq_lo, float aq_hi) {
    const int x0 = w.x1[bf][i + 1];
    const int ns = w.x1[bf][i] - x0 - 1;
    const float rn = rcpf((float)(ns + 1));
    // exactly 1 at the element's own cell, so that a thick neighbour cannot leak into it
    const float wt = x - x0 == ns ? 1.0f : (float)(x - x0 + 1) * rn;
    // interpolations (1 - w) p0 + w p1 in packed pairs; w = 1 gives p1 exactly
    const float2 w1 = make_float2(wt, wt), w0 = make_float2(1.0f - wt, 1.0f - wt);
    const float2 vbi = __ffma2_rn(w1, w.vb[bf][i], __fmul2_rn(w0, w.vb[bf][i + 1]));
    const float v = vbi.x;
    const float qds = a.qscale * w.ds[bf][i] * rn;
    const float ib = rcpf(vbi.y);
    const float ibc = ib * a.inv_chi_min;
    const float pz = kSqrtLog2e * ib;
    const float gy = v * pz, gz = (1.0f - v * (float)(1.0 / kC)) * pz;
    const float xlo = aq_lo * gz - gy, xhi = aq_hi * gz - gy;
    const float xm = xlo > 0.0f ? xlo : (xhi < 0.0f ? -xhi : 0.0f);
    const float wing = ex2f(-xm * xm);
    float Xmax = 0.0f;
#pragma unroll
    for (int k = 0; k < G; k++) {
        const float2 e = __ffma2_rn(w1, w.ln[bf][k][i], __fmul2_rn(w0, w.ln[bf][k][i + 1]));   // (eta, chi)
        const float X = fmaxf(e.y, 0.0f) * ibc;
        // (a line whose opacity is below the smallest normal float has no source here)
        const float S = e.y >= 1.17549435e-38f ? e.x * rcpf(e.y) : 0.0f;
        ln[k * kRing] = make_float4(X, X, S, S);   // line k's slot of this point
        Xmax = fmaxf(Xmax, X);
    }
    pt.a = make_float4(gz, gz, -gy, -gy);
    pt.b = make_float4(qds, qds, Xmax * wing < 1.0f ? 1.0f : 0.0f, 0.0f);
}

// Per-bin sweep state in the variables delta = dtau/sqrt 2, Phi^ = sqrt 2 Phi and
// psi^ = sqrt 2 psi, in which the recursion carries no factor 1/2:
//   s = delta_prev + delta,  Phi^ = s + Phi^_prev iota_prev,  iota = 1/(1 + delta Phi^),
//   psi^ = (s S_prev + psi^_prev) iota.
// Bins 2p and 2p+1 of a lane form pair p and are updated together with packed FP32x2
// arithmetic (fma/mul/add on float2); an odd last bin is updated alone.
template <int NB>
struct BinState {
    static constexpr int NP = NB / 2;
    static constexpr bool ODD = (NB & 1) != 0;
    float2 aq2[NP > 0 ? NP : 1], chi_p2[NP > 0 ? NP : 1], S_p2[NP > 0 ? NP : 1], d_p2[NP > 0 ? NP : 1];
    float2 Phi2[NP > 0 ? NP : 1], iota2[NP > 0 ? NP : 1], psi2[NP > 0 ? NP : 1];
    float aq1, chi_p1, S_p1, d_p1, Phi1, iota1, psi1;
    __device__ __forceinline__ float aq(int i) const {
        return i < 2 * NP ? ((i & 1) ? aq2[i >> 1].y : aq2[i >> 1].x) : aq1;
    }
    __device__ __forceinline__ void set_aq(int i, float v) {
        if (i < 2 * NP) {
            if (i & 1) aq2[i >> 1].y = v; else aq2[i >> 1].x = v;
        } else {
            aq1 = v;
        }
    }
};

__device__ __forceinline__ float2 ex2f2(const float2 t) { return make_float2(ex2f(-t.x), ex2f(-t.y)); }

// The far end of a half: the boundary row is the interior update from the virtual state
// Phi^ iota = sqrt 2, psi^ = sqrt 2 I, delta = 0.
template <int NB>
__device__ __forceinline__ void first_point(const SweepK &k, BinState<NB> &st, const float4 A, const float4 D,
                                            const float nu_g, const float v) {
    const float2 gz = make_float2(A.x, A.y), ngy = make_float2(A.z, A.w);
    const float2 X = make_float2(D.x, D.y), S = make_float2(D.z, D.w);
    const float dop = 1.0f - v * (float)(1.0 / kC);
#pragma unroll
    for (int p = 0; p < BinState<NB>::NP; p++) {
        const float2 x = __ffma2_rn(st.aq2[p], gz, ngy);
        const float2 chil = __fmul2_rn(X, ex2f2(__fmul2_rn(x, x)));
        st.chi_p2[p] = make_float2(fmaxf(chil.x, 1.0f), fmaxf(chil.y, 1.0f));
        st.S_p2[p] = __fmul2_rn(S, make_float2(fminf(chil.x, 1.0f), fminf(chil.y, 1.0f)));
        st.Phi2[p] = make_float2(kSqrt2, kSqrt2);
        st.iota2[p] = make_float2(1.0f, 1.0f);
        st.d_p2[p] = make_float2(0.0f, 0.0f);
        st.psi2[p] = make_float2(kSqrt2 * planck_k(k, nu_g * (1.0f + st.aq2[p].x * (float)(1.0 / kC)) * dop),
                                 kSqrt2 * planck_k(k, nu_g * (1.0f + st.aq2[p].y * (float)(1.0 / kC)) * dop));
    }
    if constexpr (BinState<NB>::ODD) {
        const float x = fmaf(st.aq1, gz.x, ngy.x);
        const float chil = X.x * ex2f(-x * x);
        st.chi_p1 = fmaxf(chil, 1.0f);
        st.S_p1 = S.x * fminf(chil, 1.0f);
        st.Phi1 = kSqrt2;
        st.iota1 = 1.0f;
        st.d_p1 = 0.0f;
        st.psi1 = kSqrt2 * planck_k(k, nu_g * (1.0f + st.aq1 * (float)(1.0 / kC)) * dop);
    }
}

// Update with the interval (previous point, this point); qp = (q, q) of that interval,
// A and D the point's ring entries. FLOOR = false drops the dtau floor where the caller
// knows that it cannot bind (q' >= q_nofloor): the result is the same bit for bit.
template <int NB, bool FLOOR = true>
__device__ __forceinline__ void step_point(const SweepK &k, BinState<NB> &st, const float4 A, const float4 D,
                                           const float2 qp) {
    const float2 gz = make_float2(A.x, A.y), ngy = make_float2(A.z, A.w);
    const float2 X = make_float2(D.x, D.y), S = make_float2(D.z, D.w);
#pragma unroll
    for (int p = 0; p < BinState<NB>::NP; p++) {
        const float2 x = __ffma2_rn(st.aq2[p], gz, ngy);
        const float2 chil = __fmul2_rn(X, ex2f2(__fmul2_rn(x, x)));
        const float2 chi = make_float2(fmaxf(chil.x, 1.0f), fmaxf(chil.y, 1.0f));
        const float2 Sx = __fmul2_rn(S, make_float2(fminf(chil.x, 1.0f), fminf(chil.y, 1.0f)));
        const float2 d0 = __fmul2_rn(__fadd2_rn(st.chi_p2[p], chi), qp);
        const float2 dl = FLOOR ? make_float2(fmaxf(d0.x, k.dtau_min), fmaxf(d0.y, k.dtau_min)) : d0;
        const float2 sm = __fadd2_rn(st.d_p2[p], dl);
        st.Phi2[p] = __ffma2_rn(st.Phi2[p], st.iota2[p], sm);
        const float2 den = __ffma2_rn(dl, st.Phi2[p], make_float2(1.0f, 1.0f));
        st.iota2[p] = make_float2(rcpf(den.x), rcpf(den.y));
        st.psi2[p] = __fmul2_rn(__ffma2_rn(sm, st.S_p2[p], st.psi2[p]), st.iota2[p]);
        st.d_p2[p] = dl;
        st.chi_p2[p] = chi;
        st.S_p2[p] = Sx;
    }
    if constexpr (BinState<NB>::ODD) {
        const float x = fmaf(st.aq1, gz.x, ngy.x);
        const float chil = X.x * ex2f(-x * x);
        const float chi = fmaxf(chil, 1.0f);
        const float Sx = S.x * fminf(chil, 1.0f);
        const float d0 = (st.chi_p1 + chi) * qp.x;
        const float dl = FLOOR ? fmaxf(d0, k.dtau_min) : d0;
        const float sm = st.d_p1 + dl;
        st.Phi1 = fmaf(st.Phi1, st.iota1, sm);
        st.iota1 = rcpf(fmaf(dl, st.Phi1, 1.0f));
        st.psi1 = fmaf(sm, st.S_p1, st.psi1) * st.iota1;
        st.d_p1 = dl;
        st.chi_p1 = chi;
        st.S_p1 = Sx;
    }
}

// (Phi^ iota, psi^, delta) of every bin.
template <int NB>
__device__ __forceinline__ void bin_results(const BinState<NB> &st, float (&pi)[NB], float (&ps)[NB],
                                            float (&dt)[NB]) {
#pragma unroll
    for (int p = 0; p < BinState<NB>::NP; p++) {
        const float2 pp = __fmul2_rn(st.Phi2[p], st.iota2[p]);
        pi[2 * p] = pp.x;
        pi[2 * p + 1] = pp.y;
        ps[2 * p] = st.psi2[p].x;
        ps[2 * p + 1] = st.psi2[p].y;
        dt[2 * p] = st.d_p2[p].x;
        dt[2 * p + 1] = st.d_p2[p].y;
    }
    if constexpr (BinState<NB>::ODD) {
        pi[NB - 1] = st.Phi1 * st.iota1;
        ps[NB - 1] = st.psi1;
        dt[NB - 1] = st.d_p1;
    }
}

// Sweeps half-ray r from its far end to the origin; returns per bin (Phi^ iota, psi^,
// delta) of the row next to the origin, or the empty-half values (sqrt 2, sqrt 2 I_o, 0).
// `pre` says that buffer bf already holds (or is receiving) the first window of r; on
// return it says the same of rnext (the half-ray swept next, -1 for none).
template <int G, int NB, bool SKIP>
__device__ __forceinline__ void sweep_half(const MixArgs &a, const SweepK &k, int64_t o, int l0, int grp, int r,
                                           int rnext, float nu_g, const float4 Ao, const float4 Do, RingPt *rg,
                                           float4 *rl, ElemWin<G> &w, int &bf, bool &pre, BinState<NB> &st,
                                           float (&pi)[NB], float (&ps)[NB], float (&dt)[NB], float aq_lo,
                                           float aq_hi, int &npts) {
    const int lane = threadIdx.x & 31;
    const int64_t off = a.ray_off[o * a.R + r];
    const int len = (int)(a.ray_off[o * a.R + r + 1] - off);
    int64_t offn = 0;
    int lenn = 0;
    if (rnext >= 0) {
        offn = a.ray_off[o * a.R + rnext];
        lenn = (int)(a.ray_off[o * a.R + rnext + 1] - offn);
    }
    if (len == 0) {   // an empty half is never prefetched, so `pre` is false here
#pragma unroll
        for (int i = 0; i < NB; i++) {
            pi[i] = kSqrt2;
            ps[i] = kSqrt2 * planck_k(k, nu_g * (1.0f + st.aq(i) * (float)(1.0 / kC)));
            dt[i] = 0.0f;
        }
        return;
    }
    if (!pre) {
        win_records<G>(a, off, len - 1, (int32_t)o, w, bf);
        cp_async_wait_all();
        win_gathers<G>(a, l0, w, bf);
    }
    pre = false;
    const float4 *my = rl + grp * kRing;
    int top = len - 1;         // element in window slot 0
    int xnext = -1;            // next point to stage (descending towards the origin)
    float2 qp = make_float2(0.0f, 0.0f);   // (q, q) of the interval ending at the next point
    bool first = true, far1 = false, far2 = false;
    bool fresh = true;         // first refill from this window: prefetch the next one
    do {
        if (fresh) cp_async_wait_all();
        __syncwarp();
        if (first) xnext = w.x1[bf][0] - 1;
        // Owner slot of the point of each lane. Slot i's element ends (its highest point)
        // at chunk position p_i = xnext - xcum + 1, increasing with i. The n0 slots with
        // p_i <= 0 hold or lie above xnext (the last of them holds it); the owner of
        // position j is slot n0 - 1 plus the number of slots with 1 <= p_i <= j. Slot 31
        // only precedes slot 30 and owns no point.
        const int pos = xnext - w.x1[bf][lane] + 1;
        const bool slot_ok = lane < kWin - 1 && top - lane >= 0;
        const int n0 = __popc(__ballot_sync(0xffffffffu, slot_ok && pos <= 0));
        const unsigned starts = __reduce_or_sync(0xffffffffu, (slot_ok && pos > 0 && pos < 32) ? (1u << pos) : 0u);
        const int own = n0 - 1 + __popc(starts & (0xffffffffu >> (31 - lane)));
        // points owned by slots 0 .. 30: those from xcum of slot 31 up to xnext
        const int xw = w.x1[bf][kWin - 1];
        const int cnt = min(kRing, xnext - xw + 1);
        bool my_far = false, my_tiny = false;
        if (lane < cnt) {
            RingPt pt;
            const int x = xnext - lane;
            stage_ring_point<G>(a, w, bf, own, l0, x, pt, rl + lane, aq_lo, aq_hi);
            rg[lane] = pt;
            my_far = pt.b.z != 0.0f;
            my_tiny = pt.b.x < a.q_nofloor;
        }
        const unsigned farmask = SKIP ? __ballot_sync(0xffffffffu, my_far) : 0u;
        __syncwarp();
        // On the first refill from a window, the next window: the following 31 elements of
        // this half-ray, else (this window reaches element 0) the start of the next one.
        const bool last_window = top - (kWin - 1) < 0;
        const bool issue = fresh && (!last_window || lenn > 0);
        if (fresh && !last_window) win_records<G>(a, off, top - (kWin - 1), (int32_t)o, w, bf ^ 1);
        else if (issue) win_records<G>(a, offn, lenn - 1, (int32_t)o, w, bf ^ 1);
        if (fresh && last_window) pre = issue;
        fresh = false;
        const int nb = bf ^ 1;
        auto gathers = [&]() {
            if (issue) {
                cp_async_wait_all();
                win_gathers<G>(a, l0, w, nb);
            }
        };
        int j = 0;
        if (first) {
            const float4 A = rg[0].a;
            const float vfar = -A.z / (A.x - A.z * (float)(1.0 / kC));   // v = (v pz)/pz
            first_point<NB>(k, st, A, my[0], nu_g, vfar);
            npts++;
            const float4 B = rg[0].b;
            qp = make_float2(B.x, B.y);
            far1 = false;
            far2 = false;
            j = 1;
            first = false;
        }
        // The chunk is swept in two segments, points [0, 16) and [16, cnt), with the
        // gathers of the next window issued between them (one copy of each loop body).
        // A chunk whose intervals all have q' >= q_nofloor sweeps without the dtau floor.
        const int mid = cnt < 16 ? cnt : 16;
        const bool floor_needed = __any_sync(0xffffffffu, my_tiny) || qp.x < a.q_nofloor;
        auto dense = [&](auto floor_tag, int jend) {
#pragma unroll 4
            for (; j < jend; j++) {
                step_point<NB, decltype(floor_tag)::value>(k, st, rg[j].a, my[j], qp);
                const float4 B = rg[j].b;
                qp = make_float2(B.x, B.y);
            }
        };
        if (SKIP) {
            // A point whose own and two previous points are all far changes the state by
            // O(chi_min ds) only (no-ops in FP32): rows that involve a non-floored interval
            // are still computed exactly. The points to process come from the chunk's
            // ballot of far points (bit j = point j), so skipped points cost nothing.
            const unsigned f1 = (farmask << 1) | (far1 ? 1u : 0u);                     // far(j-1)
            const unsigned f2 = (farmask << 2) | (far1 ? 2u : 0u) | (far2 ? 1u : 0u);   // far(j-2)
            const unsigned all = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
            unsigned proc = ~(farmask & f1 & f2) & all;
            if (j) proc &= ~1u;   // point 0 of the first chunk is the far end, done above
            const bool dense_chunk = (proc | (j ? 1u : 0u)) == all;
            npts += dense_chunk ? cnt - j : __popc(proc);
#pragma unroll 1
            for (int seg = 0; seg < 2; seg++) {
                if (dense_chunk) {   // nothing to skip in this chunk: the unrolled sweep
                    if (floor_needed) dense(std::true_type{}, seg ? cnt : mid);
                    else dense(std::false_type{}, seg ? cnt : mid);
                } else {
                    unsigned bits = proc & (seg ? 0xffff0000u : 0x0000ffffu);
                    while (bits) {
                        const int jj = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        float2 qprev = qp;
                        if (jj) {
                            const float4 B = rg[jj - 1].b;
                            qprev = make_float2(B.x, B.y);
                        }
                        step_point<NB>(k, st, rg[jj].a, my[jj], qprev);
                    }
                }
                if (seg == 0) gathers();
            }
            {
                const float4 B = rg[cnt - 1].b;
                qp = make_float2(B.x, B.y);
            }
            if (cnt >= 2) {
                far1 = (farmask >> (cnt - 1)) & 1u;
                far2 = (farmask >> (cnt - 2)) & 1u;
            } else {
                far2 = far1;
                far1 = farmask & 1u;
            }
        } else {
            npts += cnt - j;
#pragma unroll 1
            for (int seg = 0; seg < 2; seg++) {
                if (floor_needed) dense(std::true_type{}, seg ? cnt : mid);
                else dense(std::false_type{}, seg ? cnt : mid);
                if (seg == 0) gathers();
            }
        }
        xnext -= cnt;
        if (xnext >= 0 && xnext < xw) {   // window exhausted: move to the prefetched one
            bf = nb;
            top -= kWin - 1;
            fresh = true;
        }
    } while (xnext >= 0);
    if (pre) bf ^= 1;   // the next half-ray's first window sits in the other buffer
    step_point<NB>(k, st, Ao, Do, qp);   // the origin
    npts++;
    bin_results<NB>(st, pi, ps, dt);
}

// Per-lane, per-bin values that live across the ray pairs (slot [.][i][lane]): the pair
// sums and the backward half's result while the forward half is swept. Held in shared
// memory so that the sweeps keep their registers for the recursion.
template <int NB>
struct PairSmem {
    float acc[4][NB][32];
    float pi[NB][32], ps[NB][32], dt[NB][32];   // backward half: (Phi^ iota, psi^, delta)
};

// One work item: origin o, lines l0 .. l0+G-1, all ray pairs, all bins (one warp).
template <int G, int NB, bool SKIP>
__device__ __forceinline__ void solve_item(const MixArgs &a, int64_t o, int l0, RingPt *rg, float4 *rl,
                                           ElemWin<G> &w, PairSmem<NB> &ps) {
    constexpr int LPG = 32 / G;   // lanes per line
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPG, li = lane - grp * LPG;
    const int l = l0 + grp;
    const bool line_ok = l < a.L;
    const int lc = line_ok ? l : a.L - 1;
    const int Q = a.Q;
    const float bo = a.b[o];
    const float ibo = 1.0f / bo;
    const float2 dl = reinterpret_cast<const float2 *>(a.line)[o * a.L + lc];
    // ring entries of the origin (v = 0 there): a = (g_z, g_z, -0, -0), line = (X, X, S, S)
    const float gzo = kSqrtLog2e * ibo;
    const float Xo = fmaxf(dl.y, 0.0f) * (ibo * a.inv_chi_min);   // in units of chi_min
    const float So = dl.y > 0.0f ? dl.x / dl.y : 0.0f;
    const float4 Ao = make_float4(gzo, gzo, -0.0f, -0.0f);
    const float4 Do = make_float4(Xo, Xo, So, So);
    const float nu_g = a.nu_ghz[lc];
    const SweepK k{a.dtau_min, a.planck_a, a.planck_b};
    BinState<NB> st;
#pragma unroll
    for (int i = 0; i < NB; i++) {
        const int q = li + LPG * i;
        st.set_aq(i, q < Q ? (float)(a.roots[q] * (double)bo) : 0.0f);
        ps.acc[0][i][lane] = ps.acc[1][i][lane] = ps.acc[2][i][lane] = ps.acc[3][i][lane] = 0.0f;
    }
    // range of a_q over the whole warp (all lanes, all bins)
    float aq_lo = 1e30f, aq_hi = -1e30f;
#pragma unroll
    for (int i = 0; i < NB; i++) {
        const int q = li + LPG * i;
        if (q < Q) { aq_lo = fminf(aq_lo, st.aq(i)); aq_hi = fmaxf(aq_hi, st.aq(i)); }
    }
    for (int d = 16; d; d >>= 1) {
        aq_lo = fminf(aq_lo, __shfl_xor_sync(0xffffffffu, aq_lo, d));
        aq_hi = fmaxf(aq_hi, __shfl_xor_sync(0xffffffffu, aq_hi, d));
    }
    int bf = 0;
    bool pre = false;
    int npts = 0;   // points swept (warp-uniform), for the executed-work count
    for (int p = 0; p < a.P; p++) {
        const int rb = a.pb[p], rf = a.pf[p];
        const int rn = p + 1 < a.P ? a.pb[p + 1] : -1;
        float pif[NB], psf[NB], dtf[NB];
#pragma unroll 1
        for (int h = 0; h < 2; h++) {   // backward half, then forward half (one code copy)
            sweep_half<G, NB, SKIP>(a, k, o, l0, grp, h ? rf : rb, h ? rn : rf, nu_g, Ao, Do, rg, rl, w, bf, pre,
                                    st, pif, psf, dtf, aq_lo, aq_hi, npts);
            if (h == 0) {
#pragma unroll
                for (int i = 0; i < NB; i++) {
                    ps.pi[i][lane] = pif[i];
                    ps.ps[i][lane] = psf[i];
                    ps.dt[i][lane] = dtf[i];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const float pib = ps.pi[i][lane], psb = ps.ps[i][lane], dtb = ps.dt[i][lane];
            // the origin's line opacity, floored opacity and floored source in this bin
            const float xo = st.aq(i) * gzo;
            const float chilo = Xo * ex2f(-xo * xo);
            const float chio = fmaxf(chilo, 1.0f);
            const float Sov = So * fminf(chilo, 1.0f);
            float u, lam, uml, oml;
            if (dtb == 0.0f && dtf[i] == 0.0f) {   // isolated origin: both halves empty
                u = psb * (float)(1.0 / 1.4142135623730951); lam = 0.0f; uml = u; oml = 1.0f;
            } else {
                // sigma (Phi iota) = Phi^ iota / (delta_- + delta_+), sigma psi = psi^ / (delta_- + delta_+)
                const float sig = rcpf(dtb + dtf[i]);
                const float pi2 = pib + pif[i];
                const float iD = rcpf(fmaf(sig, pi2, 1.0f));
                const float s2 = sig * (psb + psf[i]);
                u = (Sov + s2) * iD;
                lam = iD;
                uml = s2 * iD;
                oml = sig * pi2 * iD;
            }
            const float ichi = rcpf(chio);
            ps.acc[0][i][lane] += u;
            ps.acc[1][i][lane] += lam * chilo * ichi;
            ps.acc[2][i][lane] += uml + lam * (Sov * chio - chilo * So) * ichi;
            ps.acc[3][i][lane] += oml + lam * (chio - chilo) * ichi;
        }
    }
    cp_async_wait_all();
    if (a.work && lane == 0) {
        const int lines = min(G, a.L - l0);
        atomicAdd(a.work, (unsigned long long)npts * (unsigned long long)(lines * Q));
    }
    // weighted sums over each line's bins: fixed shuffle tree in FP64 within the lane group
    const double invP = 1.0 / a.P;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < NB; i++) {
        const int q = li + LPG * i;
        const double wq = q < Q ? a.weights[q] : 0.0;
#pragma unroll
        for (int kk = 0; kk < 4; kk++) s[kk] += wq * (double)ps.acc[kk][i][lane];
        if (a.Jnu && q < Q && line_ok)
            a.Jnu[(o * a.L + l) * Q + q] = (double)ps.acc[0][i][lane] * invP * (double)kI0;
    }
#pragma unroll
    for (int kk = 0; kk < 4; kk++)
        for (int d = LPG / 2; d; d >>= 1) s[kk] += __shfl_down_sync(0xffffffffu, s[kk], d);
    if (li == 0 && line_ok) {
        a.J[o * a.L + l] = s[0] * invP * (double)kI0;
        a.Lout[o * a.L + l] = s[1] * invP;
        a.Jeff[o * a.L + l] = s[2] * invP * (double)kI0;
        a.Lc[o * a.L + l] = s[3] * invP;
    }
}

template <int G, int NB, int MINB, bool SKIP, int W>
__global__ void __launch_bounds__(32 * W, MINB) k_feautrier_warp(MixArgs a) {
    __shared__ RingPt rgs[W][kRing];
    __shared__ float4 rls[W][G * kRing];
    __shared__ ElemWin<G> ews[W];
    __shared__ PairSmem<NB> pss[W];
    const int warp = threadIdx.x >> 5;
    const int ngroups = (a.L + G - 1) / G;
    const int64_t item = (int64_t)blockIdx.x * W + warp;
    if (item >= a.n * ngroups) return;
    const int64_t o = item / ngroups;
    const int l0 = (int)(item - o * ngroups) * G;
    solve_item<G, NB, SKIP>(a, o, l0, rgs[warp], rls[warp], ews[warp], pss[warp]);
}

// Persistent variant over a batch of models: every warp takes work items (model, origin,
// line group) from a queue ordered by decreasing cost until the queue is empty. The
// per-model arguments are copied once per item into the warp's shared-memory slot.
struct BatchItem {
    int32_t model;
    int32_t local;   // origin * L + first line of the warp's line group
};

template <int G, int NB, int MINB, bool SKIP, int W>
__global__ void __launch_bounds__(32 * W, MINB)
k_feautrier_batch(const MixArgs *__restrict__ models, const BatchItem *__restrict__ items, int64_t n_items,
                  unsigned long long *counter, const int32_t *__restrict__ active) {
    __shared__ RingPt rgs[W][kRing];
    __shared__ float4 rls[W][G * kRing];
    __shared__ ElemWin<G> ews[W];
    __shared__ PairSmem<NB> pss[W];
    __shared__ MixArgs sa[W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(counter, 1ull);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= (unsigned long long)n_items) break;
        const BatchItem it = items[idx];
        if (!active[it.model]) continue;
        __syncwarp();
        if (lane == 0) sa[warp] = models[it.model];
        __syncwarp();
        const MixArgs &a = sa[warp];
        const int64_t o = it.local / a.L;
        const int l0 = (int)(it.local - o * a.L);
        solve_item<G, NB, SKIP>(a, o, l0, rgs[warp], rls[warp], ews[warp], pss[warp]);
    }
}

// Launch variants of the warp kernel: (lines per warp, bins per lane, min blocks per SM,
// far-wing skipping, warps per block).
struct WarpVariant {
    int G, NB, MINB;
    bool skip;
    int W;
    void (*fn)(MixArgs);
    void (*batch)(const MixArgs *, const BatchItem *, int64_t, unsigned long long *, const int32_t *);
};
#define MG_VARIANT_W(G, NB, M, S, W) \
    {G, NB, M, S, W, k_feautrier_warp<G, NB, M, S, W>, k_feautrier_batch<G, NB, M, S, W>}
#define MG_VARIANT(G, NB, M, S) MG_VARIANT_W(G, NB, M, S, kWarps2)
const WarpVariant kWarpVariants[] = {
    // with far-wing skipping
    MG_VARIANT(1, 1, 8, true), MG_VARIANT(1, 1, 10, true), MG_VARIANT(2, 2, 4, true), MG_VARIANT(2, 2, 5, true),
    MG_VARIANT(2, 2, 6, true), MG_VARIANT(1, 2, 4, true), MG_VARIANT(1, 2, 6, true), MG_VARIANT(1, 4, 3, true),
    MG_VARIANT(1, 4, 4, true), MG_VARIANT(2, 4, 3, true), MG_VARIANT(2, 4, 4, true), MG_VARIANT(4, 4, 3, true),
    MG_VARIANT(4, 4, 4, true),
    // the same shapes without skipping (every point swept)
    MG_VARIANT(1, 1, 8, false), MG_VARIANT(1, 1, 10, false), MG_VARIANT(2, 2, 4, false), MG_VARIANT(2, 2, 5, false),
    MG_VARIANT(2, 2, 6, false), MG_VARIANT(1, 2, 4, false), MG_VARIANT(1, 2, 6, false), MG_VARIANT(1, 4, 3, false),
    MG_VARIANT(1, 4, 4, false), MG_VARIANT(2, 4, 3, false), MG_VARIANT(2, 4, 4, false), MG_VARIANT(4, 4, 3, false),
    MG_VARIANT(4, 4, 4, false),
    // two lines x four bins per lane at 5 and 6 blocks per SM (95 and 80 registers, a few
    // spilled words) for more warps in flight on lines with 33-64 bins
    MG_VARIANT(2, 4, 5, false), MG_VARIANT(2, 4, 6, false),
    // eight bins per lane (four independent bin pairs per lane) at four lines per warp,
    // for lines with 33-64 bins; three warps per block keep the static shared memory
    // below 48 KB
    MG_VARIANT_W(4, 8, 3, false, 3), MG_VARIANT_W(4, 8, 4, false, 3), MG_VARIANT_W(4, 8, 3, true, 3),
    MG_VARIANT_W(4, 8, 4, true, 3),
};
#undef MG_VARIANT
#undef MG_VARIANT_W
constexpr int kNumWarpVariants = sizeof(kWarpVariants) / sizeof(kWarpVariants[0]);

// Far-wing skipping leaves out the floored intervals of far points. Each changes the
// sweep by O(chi_min ds), below FP32 resolution only while the floored optical depth of
// a whole ray, chi_min times the longest path through the model, is; otherwise (a large
// opacity floor) the variant's non-skipping twin runs instead.
bool skip_allowed(const mg_ctx *ctx) { return ctx->opt.chi_min * ctx->extent < 1e-7; }

int no_skip_twin(int v) {
    const WarpVariant &w = kWarpVariants[v];
    for (int u = 0; u < kNumWarpVariants; u++) {
        const WarpVariant &x = kWarpVariants[u];
        if (!x.skip && x.G == w.G && x.NB == w.NB && x.MINB == w.MINB && x.W == w.W) return u;
    }
    return v;
}

int effective_variant(const mg_ctx *ctx, int v) {
    if (v < 0 || v >= kNumWarpVariants || !kWarpVariants[v].skip || skip_allowed(ctx)) return v;
    return no_skip_twin(v);
}

bool variant_valid(int v, int L, int Q) {
    if (v < 0 || v >= kNumWarpVariants) return false;
    const WarpVariant &w = kWarpVariants[v];
    if (w.G > L) return false;
    return Q <= w.NB * (32 / w.G) && Q > (w.NB == 1 ? 0 : (w.NB / 2) * (32 / w.G));
}

}  // namespace

int mg_launch_line_data_mixed(mg_ctx *ctx) {
    const int64_t m = ctx->n * ctx->n_lines;
    MgTimed t(ctx, "line_data");
    k_line_data_f32<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(ctx->n, ctx->n_lines, ctx->n_lev,
                                                                          ctx->d_pops, ctx->d_lines, ctx->d_line,
                                                                          ctx->d_linef, ctx->d_scal + 4);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}


static void fill_args(mg_ctx *ctx, MixArgs &a) {
    const int L = ctx->n_lines, Q = ctx->Q;
    a.n = ctx->n; a.R = ctx->R; a.P = ctx->P; a.L = L; a.Q = Q;
    a.pf = ctx->d_pf; a.pb = ctx->d_pb; a.ray_off = ctx->d_ray_off; a.cells = ctx->d_cells; a.xcum = ctx->d_xcum;
    a.ds = ctx->d_dsf; a.vpar = ctx->d_vparf; a.b = ctx->d_bf; a.line = ctx->d_linef;
    a.nu_ghz = ctx->d_lconst + L;
    a.roots = ctx->d_roots; a.weights = ctx->d_weights; a.ovl_off = ctx->d_ovl_off; a.ovl = ctx->d_ovl;
    a.chi_min = (float)ctx->opt.chi_min; a.dtau_min = (float)ctx->opt.dtau_min;
    a.inv_chi_min = (float)(1.0 / ctx->opt.chi_min);
    // Every floored opacity is >= 1 in units of chi_min, so an interval with
    // q' >= q_nofloor has dtau/sqrt 2 = (chi'_prev + chi') q' >= dtau_min: the floor
    // cannot bind there.
    a.q_nofloor = std::nextafter((float)(ctx->opt.dtau_min / 2.0) * 1.000001f, INFINITY);
    a.qscale = (float)(ctx->opt.chi_min * (double)kInvSqrt8);
    a.planck_a = (float)(2.0 * kH * 1e27 / (kC * kC) / (double)kI0);
    a.planck_b = (float)(kH * 1e9 / (kKB * ctx->opt.T_cmb));
    a.J = ctx->d_J; a.Lout = ctx->d_L; a.Jeff = ctx->d_Jeff; a.Lc = ctx->d_Lc;
    a.Jnu = ctx->opt.spectrum ? ctx->d_Jnu : nullptr;
    a.kmax = (int32_t)ctx->max_pair_len;
    a.err = ctx->d_err;
    a.work = ctx->opt.profile ? ctx->d_scal + 7 : nullptr;   // executed updates, profiling runs only
    bool overlap = false;
    for (int l = 0; l < L; l++) overlap |= (ctx->h_ovl_off[l + 1] - ctx->h_ovl_off[l]) > 1;
    a.overlap = overlap;
}

static int launch_mixed(mg_ctx *ctx, int variant) {
    const int L = ctx->n_lines, Q = ctx->Q;
    bool overlap = false;
    for (int l = 0; l < L; l++) overlap |= (ctx->h_ovl_off[l + 1] - ctx->h_ovl_off[l]) > 1;
    MixArgs a{};
    fill_args(ctx, a);
    a.kmax = (int32_t)ctx->max_pair_len;
    a.overlap = overlap;
    a.err = ctx->d_err;
    size_t smem = mixed_acc_offset(a.kmax, L) + 16 * (size_t)L * Q;
    if ((overlap || Q > 128) && smem > 227 * 1024) {
        return mg_fail(ctx, MG_ERR_CAPACITY, "mixed formal solve: longest ray pair does not fit in shared memory");
    }
    int threads = 32 * std::min(L, 8);
    if (overlap) variant = -1;
    MG_CUDA(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
    if (overlap) {
        MG_CUDA(cudaFuncSetAttribute(k_feautrier_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MgTimed t(ctx, "feautrier_mixed");
        k_feautrier_mixed<true><<<(unsigned)ctx->n, threads, smem, ctx->stream>>>(a);
    } else if (variant >= 0 && variant < kNumWarpVariants) {
        const WarpVariant &wv = kWarpVariants[effective_variant(ctx, variant)];
        const int64_t items = ctx->n * ((L + wv.G - 1) / wv.G);
        const unsigned grid = (unsigned)((items + wv.W - 1) / wv.W);
        MgTimed t(ctx, "feautrier_mixed");
        wv.fn<<<grid, 32 * wv.W, 0, ctx->stream>>>(a);
    } else {
        MG_CUDA(cudaFuncSetAttribute(k_feautrier_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MgTimed t(ctx, "feautrier_mixed");
        k_feautrier_mixed<false><<<(unsigned)ctx->n, threads, smem, ctx->stream>>>(a);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

// Default launch variant for a model: two lines per warp with two bins per lane when the
// lines have <= 32 bins, otherwise one line per warp with as many bins per lane as needed.
static int default_variant(int L, int Q) {
    const int order[] = {4, 3, 2, 0, 1, 6, 5, 8, 7, 12, 11, 10, 9, 17, 16, 15, 13, 14, 19, 18, 21, 20, 25, 24, 23, 22,
                         26, 27, 28, 29, 30, 31};
    for (int v : order)
        if (variant_valid(v, L, Q)) return v;
    return -1;
}

int mg_launch_feautrier_mixed(mg_ctx *ctx) {
    int v = ctx->mixed_variant;
    if (!variant_valid(v, ctx->n_lines, ctx->Q)) v = default_variant(ctx->n_lines, ctx->Q);
    return launch_mixed(ctx, v);
}

// Autotuner: times one formal-solve launch of every valid variant on the loaded model
// (CUDA events on the context's stream, best of `reps`) and keeps the fastest.
int mg_autotune_mixed(mg_ctx *ctx, int reps, int *best, double *best_ms, int *n_tried) {
    const int L = ctx->n_lines, Q = ctx->Q;
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    int bv = -1, tried = 0;
    float bms = 1e30f;
    const int saved_profile = ctx->opt.profile;
    ctx->opt.profile = 0;
    for (int v = 0; v < kNumWarpVariants; v++) {
        if (!variant_valid(v, L, Q) || effective_variant(ctx, v) != v) continue;
        tried++;
        float vbest = 1e30f;
        for (int r = 0; r < reps + 1; r++) {
            cudaEventRecord(e0, ctx->stream);
            int rc = launch_mixed(ctx, v);
            cudaEventRecord(e1, ctx->stream);
            if (rc) { ctx->opt.profile = saved_profile; return rc; }
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < vbest) vbest = ms;   // first launch warms up
        }
        if (vbest < bms) { bms = vbest; bv = v; }
    }
    ctx->opt.profile = saved_profile;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bv >= 0) ctx->mixed_variant = bv;
    if (best) *best = bv;
    if (best_ms) *best_ms = bms;
    if (n_tried) *n_tried = tried;
    return MG_OK;
}

// ---------------------------------------------------------------- batch helpers
size_t mg_mixargs_size() { return sizeof(MixArgs); }

int mg_fill_mixargs(mg_ctx *ctx, void *out) {
    MixArgs a{};
    fill_args(ctx, a);
    if (a.overlap) return mg_fail(ctx, MG_ERR_ARG, "batch: models with overlapping lines are not batched");
    std::memcpy(out, &a, sizeof(a));
    return MG_OK;
}

int mg_variant_count() { return kNumWarpVariants; }
int mg_variant_valid(int v, int L, int Q) { return variant_valid(v, L, Q) ? 1 : 0; }
int mg_variant_effective(const mg_ctx *ctx, int v) { return effective_variant(ctx, v); }
int mg_variant_minb(int v) { return (v >= 0 && v < kNumWarpVariants) ? kWarpVariants[v].MINB : 0; }
int mg_variant_g(int v) { return (v >= 0 && v < kNumWarpVariants) ? kWarpVariants[v].G : 1; }
int mg_variant_default(int L, int Q) { return default_variant(L, Q); }

int mg_batch_launch(int v, int grid, const void *d_args, const void *d_items, int64_t n_items,
                    unsigned long long *counter, const int32_t *active, cudaStream_t stream) {
    if (v < 0 || v >= kNumWarpVariants) return MG_ERR_ARG;
    kWarpVariants[v].batch<<<grid, 32 * kWarpVariants[v].W, 0, stream>>>(static_cast<const MixArgs *>(d_args),
                                                               static_cast<const BatchItem *>(d_items), n_items,
                                                               counter, active);
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
