// Device helpers of the statistical equilibrium (eq. 'stateq', 'ourALI'), shared by the
// regular update (stateq.cu) and the allocation-free one (stateq_noalloc.cu), so that
// both assemble the same rates and solve them the same way.
#pragma once
#include "common.cuh"

namespace mg {

// Collisional de-excitation coefficient of level pair `pr` (pairs ordered (1,0), (2,0),
// (2,1), ...) at temperature Tc: linear interpolation on the tabulated grid Tg[nT],
// constant beyond its ends.
__device__ __forceinline__ double collision_k_down(const double *K, int pr, int nT, const double *Tg, double Tc) {
    const double *k = K + (size_t)pr * nT;
    if (nT == 1 || Tc <= Tg[0]) return k[0];
    if (Tc >= Tg[nT - 1]) return k[nT - 1];
    int a = 0;
    while (Tg[a + 1] < Tc) a++;
    const double w = (Tc - Tg[a]) / (Tg[a + 1] - Tg[a]);
    return k[a] + w * (k[a + 1] - k[a]);
}

// Collision rates of pair (i > j): C_ij = K_ij(T) n_coll, and the excitation rate by
// detailed balance C_ji = C_ij (g_i/g_j) exp(-(E_i - E_j)/kT).
__device__ __forceinline__ void collision_rates_pair(double kd, double ncoll, double gi, double gj, double Ei,
                                                     double Ej, double Tc, double &Cd, double &Cu) {
    Cd = kd * ncoll;
    Cu = Cd * gi / gj * exp(-(Ei - Ej) / (kKB * Tc));
}

// Radiative rates of the diagonal ALO (eq. 'ourALI') added to q[i][j] (rate i -> j):
// u -> l: A (1 - L) + B_ul Jeff, l -> u: B_lu Jeff. With `plain` the ALO is left out
// (1 - L = 1, Jeff = J): the validity fallback of Sec. 6.1. 1 - L is read directly (the
// formal solve accumulates it without cancellation).
template <int MAXLEV>
__device__ __forceinline__ void line_rates(int L, const LineConst *lc, const double *J, const double *oml,
                                           const double *Jeff, int64_t c, bool plain,
                                           double (&q)[MAXLEV][MAXLEV]) {
    for (int l = 0; l < L; l++) {
        const LineConst k = lc[l];
        const double je = plain ? J[c * L + l] : Jeff[c * L + l];
        const double om = plain ? 1.0 : oml[c * L + l];
        q[k.up][k.lo] += k.A * om + k.Bul * je;
        q[k.lo][k.up] += k.Blu * je;
    }
}

// Stationary state of the level system by Grassmann-Taksar-Heyman state reduction:
// rates q[i][j] (i -> j) are all non-negative, so every step adds non-negative terms and
// the populations come out non-negative. Returns false on a zero exit rate. (A negative
// rate, which only an ALO can produce, may give a negative or non-finite result; the
// caller's validity check catches it.)
template <int MAXLEV>
__device__ bool gth_solve(int n, double (&q)[MAXLEV][MAXLEV], double (&pi)[MAXLEV]) {
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

// Validity of a solution: every fraction finite and non-negative.
template <int MAXLEV>
__device__ __forceinline__ bool valid_fractions(int n, const double (&pi)[MAXLEV]) {
    for (int i = 0; i < n; i++)
        if (!(isfinite(pi[i]) && pi[i] >= 0.0)) return false;
    return true;
}

}  // namespace mg
