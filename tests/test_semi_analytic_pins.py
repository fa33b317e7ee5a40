"""The oracle on the paper's semi-analytic test models at the paper's own sizes (Sec. 4.1,
Table 'test_parameters': 50 shells, 12,528 cells in 3D, 192 rays, N_q = 100), against
the closed forms of eq. 'Hubble-Lemaitre3D' and eq. 'density_distribution3D'.

The 3D Hubble-Lemaitre model is a true 3D point mesh (shells of points with k-nearest
neighbour lists), so this pins the neighbour-walk tracer, the velocity-step rule and the
solver on a 3D mesh against a closed form and against the paper's accuracy claim
(relative error below 1e-4 almost everywhere)."""
import numpy as np

import synthetic as syn
from oracle import Oracle
from helpers import rel_err
import analytic as an


def _stratified_origins(m, per_band=3, bands=10, seed=0):
    """Origins from every radial band of the mesh, boundary shell excluded."""
    r = np.linalg.norm(m.pos, axis=1)
    rmax = r.max()
    rng = np.random.default_rng(seed)
    out = []
    for b in range(bands):
        sel = np.flatnonzero((r >= rmax * b / bands) & (r < rmax * (b + 1) / bands) & (m.is_bdy == 0))
        if sel.size:
            out.extend(rng.choice(sel, min(per_band, sel.size), replace=False))
    return np.sort(np.array(out, np.int64))


def test_hubble_shells_3d_paper_size_against_closed_form():
    """12,528 points on 50 shells, 192 HEALPix rays, 100 bins: the oracle's J_nu agrees
    with the closed form within 1e-4 for at least 99% of (point, bin) values, and within
    1e-3 everywhere (the largest errors sit next to the boundary shell)."""
    m = syn.hubble_shells_3d()
    assert m.n == 12_528
    o = Oracle(m, nthreads=8)
    assert o.dirs.shape[0] == 192 and o.Q == 100
    origins = _stratified_origins(m)
    _, _, _, Jnu = o.formal_solve(o.lte(), origins, spectrum=True)
    line = an.lte_line(m, o.width(0))
    Jan = an.hubble_J(m.pos[origins], o.dirs, m.meta["R"], m.meta["c_dbeta"], o.roots, line,
                      float(m.n_spec[0]))
    e = rel_err(Jnu[:, 0, :], Jan)
    assert np.quantile(e, 0.99) < 1e-4
    assert e.max() < 1e-3
    assert np.median(e) < 1e-5


def test_hubble_shells_3d_detects_a_doppler_sign_error():
    """The closed form is sensitive to the Doppler sign: evaluated with the flow
    reversed (c dbeta -> -c dbeta) it misses the oracle by more than the 1e-3 bound of
    the test above (the line is optically thin here, so J stays near the CMB and the
    sign moves it by about 1.5e-3)."""
    m = syn.hubble_shells_3d()
    o = Oracle(m, nthreads=8)
    origins = _stratified_origins(m, per_band=1)
    _, _, _, Jnu = o.formal_solve(o.lte(), origins, spectrum=True)
    line = an.lte_line(m, o.width(0))
    Jrev = an.hubble_J(m.pos[origins], o.dirs, m.meta["R"], -m.meta["c_dbeta"], o.roots, line,
                       float(m.n_spec[0]))
    assert rel_err(Jnu[:, 0, :], Jrev).max() > 1e-3


def _powerlaw(nsh, nside=4, n_q=100):
    g = dict(R_in=1e13, R=7.8e16, n_in=2e13, X=1e-6)
    m = syn.vz_problem1(abundance=g["X"], n_shells=nsh, n_q=n_q, nside=nside)
    return m, g


def test_powerlaw_sphere_192_rays_against_closed_form():
    """Power-law cloud with an empty core, 192 rays, 100 bins (eq.
    'density_distribution3D' averaged over the HEALPix directions): within 6e-2 with the
    paper's 50 shells (the paper reports errors up to ~0.4 at the steep line edges),
    and the error falls by more than 4x with 200 shells."""
    errs = {}
    for nsh in (50, 200):
        m, g = _powerlaw(nsh)
        o = Oracle(m, nthreads=8)
        r = m.pos[:, 2]
        origins = np.arange(0, nsh - 1, max(1, nsh // 12))
        _, _, _, Jnu = o.formal_solve(o.lte(), origins, spectrum=True)
        line = an.lte_line(m, o.width(0))
        Jan = an.powerlaw_J(r[origins], o.dirs, g["R_in"], g["R"], o.roots, line, g["n_in"] * g["X"])
        errs[nsh] = rel_err(Jnu[:, 0, :], Jan).max()
    assert errs[50] < 6e-2
    assert errs[200] < errs[50] / 4
