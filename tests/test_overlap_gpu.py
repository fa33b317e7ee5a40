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
