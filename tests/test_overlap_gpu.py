"""Overlapping lines: an equally spaced level ladder puts every line at the same frequency,
so each frequency bin sums the profiles of all lines (the sum over lines in the opacity
and emissivity of Sec. 2.2.1). The FP64 formal solve and one statistical-equilibrium
update against the oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle
from helpers import rel_err, gpu_context

pytestmark = pytest.mark.gpu


def test_overlapping_lines_formal_solve_and_update_fp64():
    m = syn.model_clumpy_3d(n=1500, seed=12, species=syn.species_ladder(4))
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    p0 = o.lte()
    Jo, Lo, Eo = o.formal_solve(p0)
    assert np.max(rel_err(J, Jo)) < 1e-10
    assert np.max(rel_err(E, Eo)) < 1e-10
    assert np.max(np.abs(L - Lo)) < 1e-10 * max(1e-6, float(np.max(np.abs(Lo))))
    ctx.update_populations()
    ref, nf = o.stateq(Jo, Lo, Eo)
    assert np.max(rel_err(ctx.get_populations(), ref)) < 1e-10


@pytest.mark.parametrize("n_lev", [3, 4, 5])
def test_overlapping_lines_formal_solve_mixed(n_lev):
    """The mixed-precision CTA kernel for overlapping lines (every bin sums the profiles of
    all n_lev - 1 lines of the ladder; 3 lines make the per-point line data an odd number
    of float2, the case whose accumulators once started off a 16-byte boundary): J, J_eff
    within 1e-4 relative of the oracle, L within 1e-4 of its scale; then one update."""
    m = syn.model_clumpy_3d(n=1500, seed=12, species=syn.species_ladder(n_lev))
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=1, profile=1)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    assert "feautrier_mixed" in ctx.kernel_times()
    J, L, E = ctx.get_radiation()
    Jo, Lo, Eo = o.formal_solve(o.lte())
    assert np.max(rel_err(J, Jo)) < 1e-4
    assert np.max(rel_err(E, Eo)) < 1e-4
    assert np.max(np.abs(L - Lo)) < 1e-4 * max(1e-6, float(np.max(np.abs(Lo))))
    ch, rc = ctx.update_populations()
    assert rc >= 0 and np.all(np.isfinite(ctx.get_populations()))


@pytest.mark.parametrize("n_lev", [3, 4, 5])
def test_image_overlapping_lines_fp32(n_lev):
    """Images of the ladder in a mixed-precision context: 2, 3 or 4 lines within reach of
    the channels, so the FP32 image kernel stages that many lines per point; intensities
    within 1e-4 of the oracle on sampled points."""
    m = syn.model_clumpy_3d(n=1500, seed=12, species=syn.species_ladder(n_lev))
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=1, profile=1)
    ctx.trace_rays()
    ctx.init_populations()
    origins = np.sort(np.random.default_rng(8).choice(m.n, 200, replace=False))
    u = np.linspace(-10, 10, 41) * o.width(0)
    p0 = o.lte()
    for ray in (0, 17):
        for line in (0, n_lev - 2):
            I, xy = ctx.image(ray, line, u)
            Io, _ = o.image(p0, ray, line, u, origins=origins)
            assert np.max(rel_err(I[origins], Io)) < 1e-4, (ray, line)
    assert "image_fp32" in ctx.kernel_times()
