"""Pins of the oracle's band-diagonal approximate Lambda operator (Sec. 3.4, eq. 'ALO',
'ourALI', 'ourJeff'; validity check and bandwidth reduction of Sec. 6.1).

The ALO of bandwidth b keeps the entries |k - ko| <= b of row ko of the inverse of the
discretised second-order transfer operator. The pins check that row against a dense
inverse and the identity of the constant solution, bandwidth 0 against the diagonal
ALO, the coupled rate equations against a hand-solved 2-cell closed form, and the ALI
against its fixed point (the ALO changes the path, not the fixed point)."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle, CONST
from oracle.oracle import feautrier, feautrier_row

h, kB, c = CONST["h"], CONST["kB"], CONST["c"]


def _dense_T(dtau):
    """The second-order system of Sec. 3.3 (interior rows and Auer boundary rows)."""
    K = dtau.shape[0] + 1
    T = np.zeros((K, K))
    for k in range(K):
        if k == 0:
            T[0, 0] = 1 + 2 / dtau[0] + 2 / dtau[0] ** 2; T[0, 1] = -2 / dtau[0] ** 2
        elif k == K - 1:
            T[k, k] = 1 + 2 / dtau[k - 1] + 2 / dtau[k - 1] ** 2; T[k, k - 1] = -2 / dtau[k - 1] ** 2
        else:
            a = 2 / ((dtau[k - 1] + dtau[k]) * dtau[k - 1]); cc = 2 / ((dtau[k - 1] + dtau[k]) * dtau[k])
            T[k, k - 1] = -a; T[k, k + 1] = -cc; T[k, k] = 1 + a + cc
    return T


@pytest.mark.parametrize("seed", range(6))
def test_inverse_row_vs_dense_inverse(seed):
    """Row ko of the inverse (unit-source solves read at ko) equals numpy's dense inverse
    (1e-11 relative on every entry above 1e-13 of the row's largest), and its diagonal
    equals the F/G diagonal formula of or_feautrier, a different computation."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(2, 50))
    dtau = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), K - 1))
    Tinv = np.linalg.inv(_dense_T(dtau))
    for ko in {0, K - 1, K // 2, int(rng.integers(0, K))}:
        x = feautrier_row(dtau, ko)
        ref = Tinv[ko]
        big = np.abs(ref) > 1e-13 * np.abs(ref).max()
        assert np.all(np.abs(x[big] - ref[big]) <= 1e-11 * np.abs(ref[big]))
        assert np.all(np.abs(x[~big]) <= 1e-12 * np.abs(ref).max())
        _, lam = feautrier(dtau, np.ones(K), 0.0, 0.0, ko)
        assert abs(x[ko] - lam) <= 1e-12 * lam


def test_inverse_row_sum_rule():
    """Constant S with incoming intensity S gives u = S (eq. 'GFE'), so the row's weights
    of the sources plus those of the boundary terms (2/dtau at either end) sum to one;
    every weight is positive. Also with intervals at the optical-depth floor (1e-30, a
    zero-length chord), where plain elimination of the tridiagonal matrix fails."""
    rng = np.random.default_rng(7)
    for K in (2, 3, 9, 60, 61):
        dtau = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), K - 1))
        if K == 61:
            dtau[[0, 17, 30, 59]] = 1e-30
        for ko in range(K):
            x = feautrier_row(dtau, ko)
            tot = x.sum() + x[0] * 2 / dtau[0] + x[-1] * 2 / dtau[-1]
            assert abs(tot - 1.0) <= 1e-12
            assert np.all(x > 0)


def _thick_sphere(n=40, seed=2, factor=3e3):
    m = syn.model_sphere_1d(n=n, seed=seed)
    m.n_spec = m.n_spec * factor
    return m


def test_band_zero_is_the_diagonal_alo():
    """The band formal solve's J, L and J_eff of bandwidth 0 are those of the plain formal
    solve bit for bit; the band statistical equilibrium of bandwidth 1 with every coupling
    coefficient zeroed gives the diagonal ALO's populations (same rates, one more solver)."""
    m = syn.model_clumpy_3d(n=300, seed=2)
    o = Oracle(m, nthreads=4)
    p0 = o.lte()
    J, L, E = o.formal_solve(p0)
    Jb, Lb, Eb, M = o.formal_solve_band(p0, 2)
    assert np.array_equal(J, Jb) and np.array_equal(L, Lb) and np.array_equal(E, Eb[0])
    ref, nf = o.stateq(J, L, E)
    geom = o.band_geometry(1)
    got = o.solve_band(L, E, np.zeros_like(M[..., :1]), geom, 1, p0)
    assert nf == 0 and np.max(np.abs(got - ref) / ref) < 1e-12


def test_two_cell_closed_form():
    """Two cells on a line, one ray pair, bandwidth 1: each origin's other half holds the
    other cell (weight 1), so the rate equations are
      n_u0 (R_lu0 + R_ul0) - A M01 n_u1 = n0 R_lu0,   -A M10 n_u0 + n_u1 (R_lu1 + R_ul1) = n1 R_lu1,
    with R_ul = A (1 - L) + B_ul J_eff(1) + C_ul, R_lu = B_lu J_eff(1) + C_lu and n_l = n - n_u.
    The oracle's coupled solve equals Cramer's rule on this 2x2 system; J_eff(0) - J_eff(1)
    equals the band term M A n_u(other)/(n_l B_lu - n_u B_ul)(own) of the old populations."""
    sp = syn.species_two_level(A21=1e-5)
    T = 30.0
    m = syn.model_line_1d(np.array([0.0, 2e15]), 0.0, 1e9, T, 150.0, 1e-2, sp, 21)
    o = Oracle(m)
    p0 = o.lte()
    J, L, E, M = o.formal_solve_band(p0, 1)
    geom = o.band_geometry(1)
    ca, cb, w = geom
    R = o.dirs.shape[0]
    nu = (sp.E[1] - sp.E[0]) / h
    Bul = sp.A[0] * c ** 2 / (2 * h * nu ** 3); Blu = 3 * Bul
    Cd = 2e-16 * 1e9; Cu = Cd * 3 * math.exp(-h * nu / (kB * T))
    A = sp.A[0]
    Mo = np.zeros(2)
    for o_ in range(2):
        other = 1 - o_
        for r in range(R):
            if cb[o_, r, 0] == other:
                assert w[o_, r, 0] == 1.0 and ca[o_, r, 0] == o_
                Mo[o_] += M[o_, 0, r, 0]
        assert Mo[o_] > 0
    Rul = A * (1 - L[:, 0]) + Bul * E[1][:, 0] + Cd
    Rlu = Blu * E[1][:, 0] + Cu
    n = m.n_spec
    a11, a12, a21, a22 = Rlu[0] + Rul[0], -A * Mo[0], -A * Mo[1], Rlu[1] + Rul[1]
    b1, b2 = n[0] * Rlu[0], n[1] * Rlu[1]
    det = a11 * a22 - a12 * a21
    nu0 = (b1 * a22 - a12 * b2) / det
    nu1 = (a11 * b2 - a21 * b1) / det
    got = o.solve_band(L, E[1], M, geom, 1, p0)
    assert abs(got[0, 1] - nu0) <= 1e-12 * nu0 and abs(got[1, 1] - nu1) <= 1e-12 * nu1
    assert abs(got[0, 0] - (n[0] - nu0)) <= 1e-12 * n[0]
    for o_ in range(2):
        other = 1 - o_
        band = Mo[o_] * A * p0[other, 1] / (p0[o_, 0] * Blu - p0[o_, 1] * Bul)
        assert abs((E[0][o_, 0] - E[1][o_, 0]) - band) <= 1e-12 * E[0][o_, 0]


@pytest.mark.parametrize("band", [1, 2])
def test_band_ali_reaches_the_plain_equilibrium_in_fewer_iterations(band):
    """An optically thick 1D cloud, Ng off: the ALI with the band-diagonal ALO converges to
    the same fixed point as with the diagonal one (the plain statistical equilibrium with
    J recomputed), in fewer iterations, and no bandwidth reduction is needed there."""
    m = _thick_sphere()
    o = Oracle(m, nthreads=4)
    p_d, ch_d, ok_d = o.ali(tol=1e-10, max_iter=600, ng_period=0)
    p_b, ch_b, ok_b, used = o.ali_band(band, tol=1e-10, max_iter=600, ng_period=0)
    assert ok_d and ok_b
    assert np.max(np.abs(p_b - p_d) / p_d) < 1e-8
    J, L, E = o.formal_solve(p_b)
    plain, _ = o.stateq(J, np.zeros_like(L), J)
    assert np.max(np.abs(plain - p_b) / p_b) < 1e-8
    assert len(ch_b) < len(ch_d)
    assert min(used) == band


def test_bandwidth_reduction_on_invalid_populations():
    """Validity check with bandwidth reduction (Sec. 6.1): coupling coefficients inflated so
    that the band solution has negative populations; the solve falls back to a smaller
    bandwidth and returns valid populations, those of the diagonal ALO when every band
    fails."""
    m = _thick_sphere()
    o = Oracle(m, nthreads=4)
    p0 = o.lte()
    J, L, Es, M = o.formal_solve_band(p0, 2)
    geom = o.band_geometry(2)
    pops, used, nf = o.stateq_band(J, L, Es, M, geom, 2, p0)
    assert used == 2 and np.all(pops >= 0)
    bad = M * 50.0
    assert np.any(o.solve_band(L, Es[2], bad, geom, 2, p0) < 0)
    pops, used, nf = o.stateq_band(J, L, Es, bad, geom, 2, p0)
    assert used < 2 and np.all(pops >= 0)
    if used == 0:
        ref, _ = o.stateq(J, L, Es[0])
        assert np.array_equal(pops, ref)


def test_band_ali_reduces_bandwidth_when_diverging():
    """A very optically thick 1D cloud, where the band-diagonal ALI iteration grows an
    odd-even oscillation near the empty core: the bandwidth is reduced once the change has
    grown for three iterations in a row, and the ALI converges to the same fixed point as
    with the diagonal ALO. Without the growth guard the oscillation runs on until the band
    solution has negative populations and the validity check reduces the bandwidth: more
    iterations to the same tolerance."""
    m = _thick_sphere(factor=3e5)
    o = Oracle(m, nthreads=4)
    p_d, ch_d, ok_d = o.ali(tol=1e-10, max_iter=600, ng_period=0)
    p_b, ch_b, ok_b, used = o.ali_band(1, tol=1e-10, max_iter=600, ng_period=0)
    assert ok_d and ok_b and used[0] == 1 and used[-1] == 0
    assert np.max(np.abs(p_b - p_d) / p_d) < 1e-8
    _, ch_g, ok_g, _ = o.ali_band(1, tol=1e-6, max_iter=400, ng_period=0)
    _, ch_u, ok_u, used_u = o.ali_band(1, tol=1e-6, max_iter=400, ng_period=0, grow_limit=10 ** 9)
    assert ok_g and ok_u and used_u[-1] == 0 and len(ch_g) < len(ch_u)
