"""Isotropic coherent scattering (Sec. 3.3, eq. 'GFE' with Psi+ = chi_sca J, Psi- = 0,
iterated on J) on the GPU (FP64) against the oracle: pass by pass and converged, on a
static slab and on 3D clouds with velocity fields; the slab's closed form; an ALI with
scattering step for step."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle
from helpers import rel_err, gpu_context
import paper_1912_08445_gb300 as mg
from paper_1912_08445_gb300.binding import MG_ERR_STATE, MG_ERR_ARG

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _slab(n_cells=161, chi_sca=1e-6):
    sp = syn.species_two_level(A21=1e-2)
    m = syn.model_line_1d(np.linspace(0.0, 4e6, n_cells), 0.0, 5e13, 45.0, 150.0, 1e-4, sp, 11)
    return m, np.full(n_cells, chi_sca)


def _cloud(n=200, seed=3):
    """A clumpy cloud with a radial outflow and a scattering opacity that follows the
    density (dust-like, frequency independent); it moves J by ~0.4%, in ~30 passes."""
    m = syn.model_clumpy_3d(n=n, seed=seed)
    return m, 3e-14 * m.n_coll / m.n_coll.max()


def _tiny():
    """A 20-point cloud with velocities; scattering moves J by ~8%, in ~40 passes."""
    return syn.model_tiny_3d(seed=4, n=20), np.linspace(0.0, 2e-13, 20)


CASES = {"slab": _slab, "cloud200": _cloud, "tiny": _tiny}


def test_zero_scattering_is_the_plain_formal_solve():
    m = syn.model_clumpy_3d(n=200, seed=3)
    ctx = gpu_context(m, precision=0, spectrum=1)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    Jn = ctx.get_spectrum()
    ctx.set_scattering(np.zeros(m.n), tol=1e-12, max_iter=5)
    ctx.formal_solve()
    Js, Ls, Es = ctx.get_radiation()
    assert np.array_equal(J, Js) and np.array_equal(L, Ls) and np.array_equal(E, Es)
    assert np.array_equal(Jn, ctx.get_spectrum())
    assert ctx.scattering_status() == (2, 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_scattering_passes_and_converged_match_oracle(name):
    """Three passes from no scattered light, then the converged iteration (1e-13): J, L,
    J_eff and the per-bin spectrum within 1e-10 of the oracle."""
    m, xs = CASES[name]()
    o = Oracle(m, nthreads=16)
    p0 = o.lte()
    for passes, tol in ((3, 1e-30), (4000, 1e-13)):
        ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, spectrum=1)
        ctx.trace_rays()
        ctx.init_populations()
        ctx.set_scattering(xs, tol=tol, max_iter=passes)
        ctx.formal_solve()
        J, L, E = ctx.get_radiation()
        Jn = ctx.get_spectrum()
        Jo, Lo, Eo, Jno, ch = o.formal_solve_scattering(p0, xs, tol=tol, max_iter=passes)
        assert ctx.scattering_status()[0] == len(ch), (passes, ctx.scattering_status(), len(ch))
        assert np.max(rel_err(J, Jo)) < TOL and np.max(rel_err(E, Eo)) < TOL
        assert np.max(rel_err(L, Lo, floor=1e-300)) < TOL
        assert np.max(rel_err(Jn, Jno)) < TOL


def test_slab_closed_form_on_the_gpu():
    """The two-stream closed form of the uniform slab (see the oracle's pins), per bin at
    the centre, within 1e-5 at 161 cells (second-order discretisation error ~6e-6)."""
    from test_scattering_pins import _closed_form
    m, xs = _slab()
    o = Oracle(m)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, spectrum=1)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.set_scattering(xs, tol=1e-13, max_iter=4000)
    ctx.formal_solve()
    ref = _closed_form(o, m, xs[0], 4e6)
    got = ctx.get_spectrum()[m.n // 2, 0]
    assert np.max(np.abs(got - ref) / ref) < 1e-5


def test_ali_with_scattering_matches_oracle():
    """Five ALI iterations (Ng off) with scattering, each formal solve iterated to 1e-12 and
    started from the previous one's field: populations within 1e-9 of the oracle doing the
    same steps."""
    m, xs = _tiny()
    o = Oracle(m, nthreads=16)
    pops = o.lte()
    prev = None
    for it in range(5):
        J, L, E, prev, ch = o.formal_solve_scattering(pops, xs, tol=1e-12, max_iter=4000, Jnu0=prev)
        pops, nf = o.stateq(J, L, E)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0, tol=1e-30, max_iter=5, ng_period=0)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.set_scattering(xs, tol=1e-12, max_iter=4000)
    rep, rc = ctx.iterate(allow_not_converged=True)
    assert rep["iterations"] == 5
    got = ctx.get_populations()
    big = pops >= 1e-10 * m.n_spec[:, None]
    assert np.max(rel_err(got[big], pops[big])) < 1e-9


def test_scattering_bad_calls():
    m, xs = _slab(21)
    c32 = gpu_context(m, precision=1)
    with pytest.raises(mg.MagritteError) as e:
        c32.set_scattering(xs)
    assert e.value.code == MG_ERR_STATE
    c64 = gpu_context(m, precision=0)
    bad = xs.copy(); bad[3] = -1.0
    for arr, tol, it in ((bad, 1e-8, 10), (xs, 0.0, 10), (xs, 1e-8, 0)):
        with pytest.raises(mg.MagritteError) as e:
            c64.set_scattering(arr, tol=tol, max_iter=it)
        assert e.value.code == MG_ERR_ARG
    c64.set_scattering(None)
