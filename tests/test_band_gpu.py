"""Band-diagonal approximate Lambda operator (Sec. 3.4, eq. 'ALO', 'ourALI', 'ourJeff';
validity check and bandwidth reduction of Sec. 6.1) on the GPU against the oracle, FP64:
the band terms of the formal solve and the coupled statistical equilibrium within 1e-10,
ALI iterations step for step, and iteration counts against the diagonal ALO."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle
from helpers import rel_err, gpu_context
import paper_1912_08445_gb300 as mg
from paper_1912_08445_gb300.binding import MG_ERR_ARG

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _thick_sphere(factor=3e3, n=40, seed=2):
    m = syn.model_sphere_1d(n=n, seed=seed)
    m.n_spec = m.n_spec * factor
    return m


CASES = {
    "tiny": lambda: syn.model_tiny_3d(seed=4, n=20),
    "sphere_thick": lambda: _thick_sphere(),
    "clumpy600": lambda: syn.model_clumpy_3d(n=600, seed=3),
}


def _close(got, ref, n_spec, tol=TOL):
    big = ref >= 1e-10 * n_spec[:, None]
    assert np.max(rel_err(got[big], ref[big])) < tol
    small = ~big
    if small.any():
        assert np.max(np.abs(got - ref)[small] / np.broadcast_to(n_spec[:, None], ref.shape)[small]) < 1e-14


@pytest.mark.parametrize("band", [1, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_band_terms_and_update_match_oracle(name, band):
    """From LTE: J, L, J_eff of bandwidths 0..b and every coupling coefficient within 1e-10
    of the oracle; one coupled update within 1e-10, with the same bandwidth used."""
    m = CASES[name]()
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, alo_band=band)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    Jb, M = ctx.get_band_terms()
    p0 = o.lte()
    Jo, Lo, Eo, Mo = o.formal_solve_band(p0, band)
    assert np.max(rel_err(J, Jo)) < TOL and np.max(rel_err(E, Eo[0])) < TOL
    assert np.max(rel_err(L, Lo, floor=1e-300)) < TOL
    for b in range(band):
        assert np.max(rel_err(Jb[b], Eo[b + 1], floor=1e-300)) < TOL, b
    assert np.array_equal(M == 0.0, Mo == 0.0)
    assert np.max(rel_err(M, Mo, floor=1e-300)) < TOL
    ch, rc = ctx.update_populations()
    ref, used, nf = o.stateq_band(Jo, Lo, Eo, Mo, o.band_geometry(band), band, p0)
    assert ctx.band_status()[0] == used
    _close(ctx.get_populations(), ref, m.n_spec)


@pytest.mark.parametrize("band", [1, 2])
def test_band_ali_iterations_match_oracle(band):
    """Eight ALI iterations with the band ALO (Ng off) step for step against the oracle's
    band ALI: populations within 1e-9 (the coupled solve's residual carries over)."""
    m = _thick_sphere(factor=3e4)
    o = Oracle(m, nthreads=16)
    ref, ch, conv, used = o.ali_band(band, tol=1e-30, max_iter=8, ng_period=0)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, alo_band=band, tol=1e-30, max_iter=8, ng_period=0)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate(allow_not_converged=True)
    assert rep["iterations"] == 8 and rep["alo_band"] == used[-1]
    _close(ctx.get_populations(), ref, m.n_spec, tol=1e-9)


def test_band_ali_fixed_point_and_iteration_counts():
    """A thick 1D cloud and a thick 3D cloud: the band ALI converges to the diagonal ALI's
    fixed point (1e-9), in the oracle's number of iterations, and in fewer iterations than
    the diagonal ALO."""
    for m, bands in ((_thick_sphere(factor=3e4), (1, 2)),
                     (syn.model_clumpy_3d(n=400, seed=3), (1, 2))):
        m.n_spec = m.n_spec * (1.0 if m.name == "sphere1d" else 30.0)
        o = Oracle(m, nthreads=16)
        its = {}
        pops = {}
        for band in (0,) + bands:
            ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, alo_band=band, tol=1e-6, max_iter=400, ng_period=0)
            ctx.trace_rays()
            ctx.init_populations()
            rep, rc = ctx.iterate()
            its[band] = rep["iterations"]
            pops[band] = ctx.get_populations()
            if band:
                _, ch, conv, used = o.ali_band(band, tol=1e-6, max_iter=400, ng_period=0)
                assert conv and len(ch) == its[band], (m.name, band)
        for band in bands:
            assert its[band] < its[0], (m.name, its)
            _close(pops[band], pops[0], m.n_spec, tol=1e-4)


def test_band_ali_reduces_bandwidth_when_diverging():
    """The very thick 1D cloud whose band iteration grows an odd-even oscillation: the
    bandwidth in use drops to 0 after three growing changes, and the ALI converges to the
    diagonal ALO's fixed point in the oracle's number of iterations."""
    m = _thick_sphere(factor=3e5)
    o = Oracle(m, nthreads=16)
    pd, chd, okd = o.ali(tol=1e-8, max_iter=600, ng_period=0)
    pb, chb, okb, used = o.ali_band(1, tol=1e-8, max_iter=600, ng_period=0)
    assert okd and okb and used[-1] == 0
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, alo_band=1, tol=1e-8, max_iter=600, ng_period=0)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate()
    assert rep["converged"] and rep["alo_band"] == 0 and rep["iterations"] == len(chb)
    _close(ctx.get_populations(), pd, m.n_spec, tol=1e-6)


def test_band_ali_with_ng_reaches_the_fixed_point():
    """Band ALO with Ng acceleration (every 4th iteration) converges to the same fixed
    point as the oracle's band ALI with Ng, in the same number of iterations."""
    m = _thick_sphere(factor=3e4)
    o = Oracle(m, nthreads=16)
    ref, ch, conv, used = o.ali_band(1, tol=1e-8, max_iter=400, ng_period=4)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, alo_band=1, tol=1e-8, max_iter=400, ng_period=4)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate()
    assert conv and rep["converged"] and abs(rep["iterations"] - len(ch)) <= 1
    _close(ctx.get_populations(), ref, m.n_spec, tol=1e-7)


def test_band_alo_needs_fp64():
    with pytest.raises(mg.MagritteError) as e:
        mg.Context(precision=1, alo_band=1)
    assert e.value.code == MG_ERR_ARG
    with pytest.raises(mg.MagritteError):
        mg.Context(precision=0, alo_band=3)
