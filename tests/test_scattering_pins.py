"""Pins of the oracle's scattering (Sec. 2.1 eq. 'RTE', Sec. 3.3 eq. 'RTE2', 'GFE'):
isotropic, coherent scattering with a frequency-independent opacity chi_sca, for which
Psi- = 0 and Psi+ = chi_sca J, iterated on J as Sec. 3.3 prescribes.

The closed form: on one ray pair through a uniform static slab (the paper's 1D setup of
two rays), J = u, so the source is S = eps S_l + (1 - eps) u with
eps = chi_l phi / (chi_l phi + chi_sca) per bin, and u'' = eps (u - S_l) in the total
optical depth; with incoming intensity I at both faces,
    u(tau) = S_l + (I - S_l) cosh(sqrt(eps) (tau - T/2)) / (cosh(sqrt(eps) T/2) + sqrt(eps) sinh(sqrt(eps) T/2)).
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle, CONST, planck

h, kB, c = CONST["h"], CONST["kB"], CONST["c"]


def _slab(n_cells, chi_sca, n_h2=5e13, abundance=1e-4, T=45.0, L=4e6, n_q=11):
    sp = syn.species_two_level(A21=1e-2)
    m = syn.model_line_1d(np.linspace(0.0, L, n_cells), 0.0, n_h2, T, 150.0, abundance, sp, n_q)
    return m, np.full(n_cells, chi_sca)


def _closed_form(o, m, chi_sca, L):
    """Per bin of the centre cell: the two-stream solution at the slab's centre."""
    sp = m.species
    pops = o.lte()
    nu = (sp.E[1] - sp.E[0]) / h
    Bul = sp.A[0] * c ** 2 / (2 * h * nu ** 3); Blu = sp.g[1] / sp.g[0] * Bul
    pre = h * nu / (4 * math.pi)
    eta = pre * pops[0, 1] * sp.A[0]
    chi = pre * (pops[0, 0] * Blu - pops[0, 1] * Bul)
    Sl = eta / chi
    b = o.width(0)
    dnu = nu * b / c
    out = []
    for r in o.roots:
        phi = math.exp(-r * r) / (dnu * math.sqrt(math.pi))
        ct = chi * phi + chi_sca
        eps = chi * phi / ct
        tc = ct * L / 2
        I = planck(nu * (1 + r * b / c), 2.725)
        se = math.sqrt(eps)
        out.append(Sl + (I - Sl) / (math.cosh(se * tc) + se * math.sinh(se * tc)))
    return np.array(out)


def test_zero_scattering_is_the_plain_formal_solve():
    """chi_sca = 0 gives the plain formal solution bit for bit, in one iteration."""
    m = syn.model_clumpy_3d(n=300, seed=2)
    o = Oracle(m, nthreads=4)
    p0 = o.lte()
    J, L, E, Jnu = o.formal_solve(p0, spectrum=True)
    Js, Ls, Es, Jnus, ch = o.formal_solve_scattering(p0, np.zeros(m.n), tol=1e-12, max_iter=3)
    assert np.array_equal(J, Js) and np.array_equal(L, Ls) and np.array_equal(E, Es) and np.array_equal(Jnu, Jnus)
    assert ch[-1] == 0.0 and len(ch) == 2


@pytest.mark.parametrize("chi_sca", [1e-7, 1e-6])
def test_slab_closed_form_second_order(chi_sca):
    """Uniform static slab, one ray pair, line and scattering opacities comparable at the
    line centre and pure scattering in the wings (total optical half-thickness ~0.2-4):
    the converged per-bin mean intensity at the centre, which the scattering moves by
    tens of percent, approaches the closed form at second order in the cell size (errors
    fall ~4x per halving)."""
    L = 4e6
    errs = []
    for n in (41, 81, 161):
        m, xs = _slab(n, chi_sca, L=L)
        o = Oracle(m, nthreads=4)
        J, Lw, E, Jnu, ch = o.formal_solve_scattering(o.lte(), xs, tol=1e-13, max_iter=4000)
        assert ch[-1] < 1e-13
        ref = _closed_form(o, m, chi_sca, L)
        errs.append(np.max(np.abs(Jnu[n // 2, 0] - ref) / ref))
        # the scattering matters: without it (first pass, no scattered light) far off
        Jn0 = o.formal_solve_scattering(o.lte(), xs, tol=1e-30, max_iter=1)[3]
        assert np.max(np.abs(Jn0[n // 2, 0] - ref) / ref) > 0.05
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-3 and all(1.7 < r < 2.3 for r in rates), (errs, rates)


def test_scattering_wrong_sign_or_factor_misses_the_closed_form():
    """The closed form separates scattering from absorption: the same slab with the
    scattering opacity turned into pure absorption (no re-emission) misses it by far."""
    L, n, chi_sca = 4e6, 161, 1e-6
    m, xs = _slab(n, chi_sca, L=L)
    o = Oracle(m, nthreads=4)
    ref = _closed_form(o, m, chi_sca, L)
    J, Lw, E, Jnu, ch = o.formal_solve_scattering(o.lte(), xs, tol=1e-30, max_iter=1)   # first pass: J_prev = 0
    assert np.max(np.abs(Jnu[n // 2, 0] - ref) / ref) > 1e-2


def test_pure_scattering_limit_carries_the_boundary_radiation():
    """With no line emission in the slab (a species density so low that the line is
    negligible) and strong scattering, the mean intensity everywhere tends to the
    incoming radiation (conservative scattering of the CMB)."""
    m, xs = _slab(41, 1e-6, abundance=1e-20, L=4e6)
    o = Oracle(m, nthreads=4)
    J, Lw, E, Jnu, ch = o.formal_solve_scattering(o.lte(), xs, tol=1e-12, max_iter=20000)
    nu = (m.species.E[1] - m.species.E[0]) / h
    I = planck(nu * (1 + o.roots * o.width(0) / c), 2.725)
    assert np.max(np.abs(Jnu[:, 0, :] - I[None, :]) / I[None, :]) < 1e-6
