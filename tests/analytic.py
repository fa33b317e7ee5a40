"""Closed forms of the paper's semi-analytic tests (Sec. 4.1), vectorised with numpy.

Both models hold LTE populations, so the line source function S is constant and the
mean intensity is J_nu = S + <(B_nu - S) exp(-tau_nu)> over the directions (eq.
'J_for_constant_S'). With the discrete directions of a model the angle integral is the
plain average over those directions, as in the formal solve itself (uniform weights).
The boundary intensity is the CMB at the comoving frequency where a ray enters the
model, the reading the formal solve uses (a 5e-6 effect in the Hubble test)."""
import math

import numpy as np
from scipy.special import erf

H = 6.62607015e-34
KB = 1.380649e-23
C = 299792458.0
T_CMB = 2.725


def planck(nu, T):
    return 2.0 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (KB * T))


def lte_line(model, width):
    """Line frequency, constant source function and line-integrated opacity of the
    2-level species at LTE (eq. 'lines' with the Boltzmann populations), and the
    Doppler width delta_nu = nu b / c of the cell width b (m/s)."""
    sp = model.species
    T = float(model.T[0])
    nu = (sp.E[1] - sp.E[0]) / H
    Bul = sp.A[0] * C ** 2 / (2 * H * nu ** 3)
    Blu = sp.g[1] / sp.g[0] * Bul
    w = sp.g * np.exp(-(sp.E - sp.E[0]) / (KB * T))
    frac = w / w.sum()
    pre = H * nu / (4 * math.pi)
    eta_per_n = pre * frac[1] * sp.A[0]
    chi_per_n = pre * (frac[0] * Blu - frac[1] * Bul)
    return dict(nu=nu, S=eta_per_n / chi_per_n, chi_per_n=chi_per_n, dnu=nu * width / C)


def hubble_J(pos, dirs, R, c_dbeta, roots, line, n_spec):
    """Mean intensity [n_points][Q] of the homogeneous Hubble-Lemaitre sphere (eq.
    'Hubble-Lemaitre3D' with the optical depth of eq. 'optical_depth'): along direction
    n the distance to the boundary sphere is l = -x.n + sqrt(R^2 - |x|^2 + (x.n)^2), and
    tau = chi/(2 nu dbeta) (erf((nu - nu_l)/dnu) - erf((nu (1 - dbeta l) - nu_l)/dnu)).
    A single ray pair along +-z through points on the z axis is the 1D model (eq.
    'Hubble-Lemaitre1D')."""
    nu_l, S, dnu = line["nu"], line["S"], line["dnu"]
    chi = line["chi_per_n"] * n_spec
    dbeta = c_dbeta / C
    nu = nu_l + np.asarray(roots)[None, :, None] * dnu                  # [1][Q][1]
    xd = -(pos @ dirs.T)                                                  # [n][R]
    r2 = np.sum(pos * pos, axis=1)[:, None]
    ell = (xd + np.sqrt(np.maximum(R * R - r2 + xd * xd, 0.0)))[:, None, :]   # [n][1][R]
    tau = chi / (2 * nu * dbeta) * (erf((nu - nu_l) / dnu) - erf((nu * (1 - dbeta * ell) - nu_l) / dnu))
    B = planck(nu * (1 - dbeta * ell), T_CMB)
    return S + np.mean((B - S) * np.exp(-tau), axis=2)


def powerlaw_J(r, dirs, R_in, R, roots, line, n_spec_in):
    """Mean intensity [n_points][Q] of the power-law cloud n = n_in (R_in/r)^2 with an
    empty core (Sec. 4.1.2) at points on the +z axis at radii r, without velocities.
    For the angle theta between a direction and the inward radial, with impact parameter
    p = r sin(theta), tau = chi_in phi R_in^2 / p (pi/2 - theta + arccos(p/R) - f), with
    f = 2 arccos(p/R_in) for rays that cross the core (theta < arcsin(R_in/r)); the radial
    limits p -> 0 are chi_in phi R_in^2 (1/r - 1/R) outwards and
    chi_in phi R_in^2 (2/R_in - 1/r - 1/R) inwards through the core."""
    nu_l, S, dnu = line["nu"], line["S"], line["dnu"]
    roots = np.asarray(roots)
    phi = np.exp(-roots ** 2) / (dnu * math.sqrt(math.pi))             # [Q]
    k0 = line["chi_per_n"] * n_spec_in * phi * R_in ** 2                # [Q]
    r = np.asarray(r, np.float64)[:, None]                              # [n][1]
    cth = np.clip(-dirs[:, 2], -1.0, 1.0)[None, :]                      # [1][R]
    th = np.arccos(cth)
    p = r * np.sin(th)
    radial = p < 1e-9 * r
    ps = np.where(radial, 1.0, p)
    core = (p < R_in) & (cth > 0)
    f = np.where(core, 2 * np.arccos(np.minimum(ps / R_in, 1.0)), 0.0)
    g = (math.pi / 2 - th + np.arccos(np.minimum(ps / R, 1.0)) - f) / ps
    g = np.where(radial, np.where(cth > 0, 2 / R_in - 1 / r - 1 / R, 1 / r - 1 / R), g)   # [n][R]
    tau = k0[None, :, None] * g[:, None, :]                             # [n][Q][R]
    B = planck(nu_l + roots * dnu, T_CMB)[None, :, None]
    return S + np.mean((B - S) * np.exp(-tau), axis=2)
