"""The allocation-free statistical-equilibrium update (mg_update_populations_noalloc),
for callers that cannot allocate device memory when they update populations, gives the
same populations and convergence measure as mg_update_populations, on two calls in a
row, without allocating and without touching the context's own populations.

Kept in a file that pytest collects last, so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest

import synthetic as syn
from helpers import rel_err, gpu_context

pytestmark = pytest.mark.gpu


def test_noalloc_update_matches_existing_entry_point():
    import torch
    m = syn.model_sphere_1d(n=120, seed=2)
    m.n_spec = m.n_spec * 3e3
    ctx = gpu_context(m)
    ctx.trace_rays()
    ctx.init_populations()
    n, lev = m.n, m.species.n_lev
    d_old = torch.empty((n, lev), dtype=torch.float64, device="cuda")
    d_new = torch.empty_like(d_old)
    for call in range(2):
        ctx.formal_solve()
        ctx.get_populations_dev(d_old.data_ptr())
        before = ctx.get_populations()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ch_na, nf_na, rc_na = ctx.update_populations_noalloc(d_old.data_ptr(), d_new.data_ptr())
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:   # kernels and the static scratch are resident after the first call
            assert free1 == free0
        # the variant leaves the context's populations alone
        assert np.array_equal(ctx.get_populations(), before)
        ch, rc = ctx.update_populations()      # the existing entry point advances the context
        ref = ctx.get_populations()
        got = d_new.cpu().numpy()
        assert np.max(rel_err(got, ref)) < 1e-10
        assert abs(ch_na - ch) <= 1e-10 * ch
        assert rc_na == rc and nf_na == 0
