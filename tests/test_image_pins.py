"""The oracle's images (Sec. 3.5, 'Imaging the model') pinned to closed forms.

An image along direction n holds, for every model point, the intensity leaving the model
along n on the ray pair through that point, carried with the first-order transfer
equation dI/dtau = S - I (linear source between points, Olson & Kunasz 1987), at
channel frequencies nu_l (1 + u/c) in the model's rest frame, placed at the point's
projection on the plane orthogonal to n."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erf

import synthetic as syn
from oracle import Oracle, first_order
from helpers import rel_err
import analytic as an

C = an.C


def _linear_exact(T, a, b, I0):
    """I(T) for dI/dt = a + b t - I, I(0) = I0."""
    return I0 * math.exp(-T) + a * (-math.expm1(-T)) + b * (T + math.expm1(-T))


@pytest.mark.parametrize("scale", [1e-12, 1e-4, 0.3, 5.0])
def test_first_order_exact_for_linear_source(scale):
    """A source linear in tau is integrated exactly at any step size (the Taylor branch
    below 1e-3 included), and the direction matters: the reversed point order gives the
    closed form of the reversed source instead."""
    rng = np.random.default_rng(int(scale * 1e3) + 1)
    dt = rng.uniform(0.2, 1.0, 40) * scale
    t = np.concatenate([[0.0], np.cumsum(dt)])
    T = float(t[-1])
    a, b, I0 = 2.0, 0.7 / T, 0.3
    got = first_order(dt, a + b * t, I0)
    assert abs(got - _linear_exact(T, a, b, I0)) <= 1e-13 * abs(_linear_exact(T, a, b, I0))
    rev = first_order(dt[::-1], (a + b * t)[::-1], I0)
    assert abs(rev - _linear_exact(T, a + b * T, -b, I0)) <= 1e-13 * abs(rev)
    if scale >= 0.3:
        assert abs(rev - got) > 1e-3 * abs(got)


def test_first_order_floored_opacity_keeps_emission():
    """Where the opacity is floored, S = eta/chi_min is huge and dtau = chi_min ds tiny:
    the step still adds eta ds (the Taylor weights carry no cancellation)."""
    chi_min, eta, ds = 1e-30, 1e-20, 1e10
    S = np.full(5, eta / chi_min)
    dt = np.full(4, chi_min * ds)
    got = first_order(dt, S, 1.0)
    assert abs(got - (1.0 + 4 * eta * ds)) < 1e-12


def test_first_order_second_order_convergence():
    """Smooth non-linear source S = 1 + sin(3t) over tau in [0, 4]: against the exact
    integral the error falls by about 4x per halving of the step."""
    Sf = lambda t: 1.0 + math.sin(3 * t)
    T = 4.0
    exact = 0.5 * math.exp(-T) + quad(lambda t: Sf(t) * math.exp(-(T - t)), 0, T, epsabs=1e-14)[0]
    err = []
    for K in (40, 80, 160):
        t = np.linspace(0, T, K + 1)
        err.append(abs(first_order(np.diff(t), [Sf(x) for x in t], 0.5) - exact))
    assert err[1] < err[0] / 3.5 and err[2] < err[1] / 3.5


def _channels(b, k=8.0, n=33):
    return np.linspace(-k, k, n) * b


def test_image_constant_source_slab():
    """Static uniform slab (the Hubble line model without flow, 1e6 times denser): every
    point of the line sees the same outward intensity S + (B - S) exp(-tau), tau up to
    180, to rounding."""
    m = syn.hubble_line_1d(n_cells=100, c_dbeta=0.0, n_q=31)
    m.n_spec = m.n_spec * 1e6
    o = Oracle(m, nthreads=8)
    b = o.width(0)
    u = _channels(b, 4.0, 17)
    I, xy = o.image(o.lte(), 0, 0, u)
    line = an.lte_line(m, b)
    chi = line["chi_per_n"] * float(m.n_spec[0])
    phi = np.exp(-(u / b) ** 2) / (line["dnu"] * math.sqrt(math.pi))
    tau = chi * phi * 2 * 495e3
    nu = line["nu"] * (1 + u / C)
    Ian = line["S"] + (an.planck(nu, an.T_CMB) - line["S"]) * np.exp(-tau)
    assert tau.max() > 100
    assert rel_err(I, Ian[None, :]).max() < 1e-12
    assert np.allclose(xy, 0.0, atol=1e-9)   # all points lie on the line of sight


def _hubble_line_image(m, o, u, R, c_dbeta):
    """Outward intensity along +z of the Hubble-Lemaitre line (Sec. 4.1.1) in the rest
    frame: w = c dbeta z, tau = chi/(2 nu dbeta)(erf((nu(1 + dbeta R) - nu_l)/dnu) -
    erf((nu(1 - dbeta R) - nu_l)/dnu)), entering at z = -R with the CMB at nu (1 + dbeta R)."""
    line = an.lte_line(m, o.width(0))
    chi = line["chi_per_n"] * float(m.n_spec[0])
    db = c_dbeta / C
    nu = line["nu"] * (1 + u / C)
    b = o.width(0)
    # (nu (1 -+ db R) - nu_l)/dnu written without the cancellation of nu - nu_l
    xp = (u * (1 + db * R) + C * db * R) / b
    xm = (u * (1 - db * R) - C * db * R) / b
    tau = chi / (2 * nu * db) * (erf(xp) - erf(xm))
    return line["S"] + (an.planck(nu * (1 + db * R), an.T_CMB) - line["S"]) * np.exp(-tau), tau


@pytest.mark.parametrize("boost", [1.0, 1e4])
def test_image_hubble_line_closed_form(boost):
    """Hubble-Lemaitre line, thin (the paper's model) and 1e4 times denser: the image of
    every point matches the closed form (2e-6 thin; 5e-3 with tau up to 0.3, where the
    line emission is 100 times the CMB), and refining the grid 4x cuts the error by more
    than 10x (second order: 16x measured)."""
    errs = {}
    for nc in (100, 400):
        m = syn.hubble_line_1d(n_cells=nc, n_q=31)
        m.n_spec = m.n_spec * boost
        o = Oracle(m, nthreads=8)
        u = _channels(o.width(0))
        I, _ = o.image(o.lte(), 0, 0, u, origins=np.array([0, nc // 3, nc - 1]))
        Ian, tau = _hubble_line_image(m, o, u, 495e3, 0.01)
        errs[nc] = rel_err(I, Ian[None, :]).max()
    assert errs[100] < (2e-6 if boost == 1.0 else 5e-3)
    assert errs[400] < errs[100] / 10


def test_image_lattice_axis_flow():
    """9^3 cubic lattice with a flow along z (v = c dbeta z, 1.25 km/s per cell against a
    width of 0.6 km/s), lines of sight along the lattice axis through interior columns:
    every column's image matches the closed form of the line (peak optical depth 12)
    within the velocity sampling's error, 5e-2 at the default step of 1/3 width, and 8x
    smaller at 1/12 (the inserted points resolve the profile at second order)."""
    mm, sp = 9, 1e12
    m = syn.model_lattice_3d(m=mm, spacing=sp)
    m.dirs = np.array([[0, 0, 1.0], [0, 0, -1.0]])
    L = (mm - 1) * sp
    c_dbeta = 1e4 / L
    m.vel = np.zeros_like(m.pos)
    m.vel[:, 2] = c_dbeta * m.pos[:, 2]
    line = an.lte_line(m, Oracle(m).width(0))
    phi0 = 1.0 / (line["dnu"] * math.sqrt(math.pi))
    m.n_spec = np.full(m.n, 12.0 / (line["chi_per_n"] * phi0 * L))
    ijk = np.stack(np.meshgrid(np.arange(mm), np.arange(mm), np.arange(mm), indexing="ij"), -1).reshape(-1, 3)
    cols = np.flatnonzero((ijk[:, 0] > 0) & (ijk[:, 0] < mm - 1) & (ijk[:, 1] > 0) & (ijk[:, 1] < mm - 1))
    errs = {}
    for f in (1.0 / 3.0, 1.0 / 12.0):
        o = Oracle(m, nthreads=8, dshift_frac=f)
        u = _channels(o.width(0), 12.0, 49)
        I, xy = o.image(o.lte(), 0, 0, u, origins=cols)
        Ian, tau = _hubble_line_image(m, o, u, L / 2, c_dbeta)
        assert tau.max() > 1.0
        errs[f] = rel_err(I, Ian[None, :]).max()
        assert np.ptp(I, axis=0).max() <= 1e-12 * I.max()   # every column alike
    assert errs[1.0 / 3.0] < 5e-2
    assert errs[1.0 / 12.0] < errs[1.0 / 3.0] / 8
    # the projection keeps the lattice's x, y coordinates up to a rotation in the plane
    assert np.allclose(np.sum(xy ** 2, 1), np.sum(m.pos[cols, :2] ** 2, 1), rtol=1e-12, atol=1e-6 * sp ** 2)


def test_image_projection_is_orthonormal():
    """xy are coordinates in an orthonormal basis of the plane orthogonal to n:
    |xy|^2 + (x.n)^2 = |x|^2 for every point and direction, and distances between points
    within the plane are kept."""
    m = syn.model_clumpy_3d(n=600, seed=5)
    o = Oracle(m, nthreads=8)
    pops = o.lte()
    orig = np.arange(0, m.n, 7)
    for r in (0, 5, 17, 47):
        n = o.dirs[r]
        _, xy = o.image(pops, r, 0, np.zeros(1), origins=orig)
        x = m.pos[orig]
        assert np.allclose(np.sum(xy ** 2, 1) + (x @ n) ** 2, np.sum(x * x, 1), rtol=1e-12)
        d = x[1:] - x[:-1]
        dp = d - np.outer(d @ n, n)
        assert np.allclose(np.sum((xy[1:] - xy[:-1]) ** 2, 1), np.sum(dp * dp, 1), rtol=1e-10)


def test_image_hubble_shells_3d_paper_model():
    """The paper's 3D Hubble-Lemaitre mesh (12,528 points): per line of sight the closed
    form has the chord through the sphere, the walk ends at boundary points near it; the
    median error over points and channels is 1e-5, and 99% are within 2e-3."""
    m = syn.hubble_shells_3d()
    o = Oracle(m, nthreads=8)
    b = o.width(0)
    u = _channels(b)
    orig = np.sort(np.random.default_rng(3).choice(m.n, 300, replace=False))
    line = an.lte_line(m, b)
    chi = line["chi_per_n"] * float(m.n_spec[0])
    db = m.meta["c_dbeta"] / C
    R = m.meta["R"]
    for r in (0, 77):
        n = o.dirs[r]
        I, _ = o.image(o.lte(), r, 0, u, origins=orig)
        x = m.pos[orig]
        h = np.sqrt(np.maximum(R * R - (np.sum(x * x, 1) - (x @ n) ** 2), 0.0))[:, None]
        nu = line["nu"] * (1 + u / C)[None, :]
        xp = (u[None, :] * (1 + db * h) + C * db * h) / b
        xm = (u[None, :] * (1 - db * h) - C * db * h) / b
        tau = chi / (2 * nu * db) * (erf(xp) - erf(xm))
        Ian = line["S"] + (an.planck(nu * (1 + db * h), an.T_CMB) - line["S"]) * np.exp(-tau)
        e = rel_err(I, Ian)
        assert np.median(e) < 1e-5
        assert np.quantile(e, 0.99) < 2e-3
