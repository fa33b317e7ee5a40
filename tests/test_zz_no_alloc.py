"""The allocation-free statistical-equilibrium update (mg_update_populations_noalloc).

Some callers of this library cannot allocate device memory at the moment they update
level populations: a framework whose allocator owns the GPU's memory, a loop that cannot
take the synchronisation an allocation may cause, or a process with a fixed memory
budget. For them the update keeps its scratch in a static device array and takes the
populations as caller-owned device buffers. These tests check that it gives the same
populations, fallback count and convergence measure as the oracle and as
mg_update_populations, on two calls in a row, without allocating (the first call
included: the set-up that may allocate is done when the species is set), and that it
refuses bad calls.

Kept in a file that pytest collects last, so that a run stopping at the first failure
has already run every other test."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle, CONST
from helpers import rel_err, gpu_context
import paper_1912_08445_gb300 as mg
from paper_1912_08445_gb300.binding import MG_ERR_ARG, MG_ERR_STATE, MG_ERR_CAPACITY, MG_WARN_NEG_POP_FALLBACK

pytestmark = pytest.mark.gpu
h, kB, c = CONST["h"], CONST["kB"], CONST["c"]


def _model(name):
    if name == "two_level_300":
        return syn.model_sphere_1d(n=300, seed=5)
    if name == "rotor5_1500":
        return syn.model_clumpy_3d(n=1500, seed=6)
    if name == "rotor20_1000":
        return syn.model_disc(n=1000, seed=3, nside=1, n_q=31)
    raise KeyError(name)


def _push_below_zero(m, J, L, cells):
    """J_eff of the given cells of a 2-level model such that the excitation rate is
    -C_lu/2: their ALO solution has a negative upper population (validity fallback)."""
    sp = m.species
    nu = (sp.E[1] - sp.E[0]) / h
    Blu = sp.g[1] / sp.g[0] * sp.A[0] * c ** 2 / (2 * h * nu ** 3)
    E = J.copy()
    for cc in cells:
        Cu = float(sp.K_down[0, 0]) * m.n_coll[cc] * sp.g[1] / sp.g[0] * math.exp(-h * nu / (kB * m.T[cc]))
        E[cc, 0] = -1.5 * Cu / Blu
    return E


def _close_to_oracle(got, ref, n_spec):
    """Levels holding at least 1e-10 of the cell's species (those the convergence measure
    counts) within 1e-10 relative; the rest within 1e-14 of the cell's species density,
    since the oracle's LU solve resolves populations only down to rounding of the cell
    total (it returns values near -1e-16 n for levels near 1e-30 n of a 20-level rotor,
    where GTH keeps them positive)."""
    big = ref >= 1e-10 * n_spec[:, None]
    assert np.max(rel_err(got[big], ref[big])) < 1e-10
    assert np.max(np.abs(got - ref)[~big] / np.broadcast_to(n_spec[:, None], ref.shape)[~big], initial=0.0) < 1e-14


@pytest.mark.parametrize("name", ["two_level_300", "rotor5_1500", "rotor20_1000"])
def test_noalloc_update_matches_oracle_and_existing_entry_point(name):
    import torch
    m = _model(name)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=0)
    ctx.trace_rays()
    ctx.init_populations()
    n, lev = m.n, m.species.n_lev
    d_old = torch.empty((n, lev), dtype=torch.float64, device="cuda")
    d_new = torch.empty_like(d_old)
    for call in range(2):
        ctx.formal_solve()
        J, L, E = ctx.get_radiation()
        fallback = name == "two_level_300"
        if fallback:   # cells that must take the validity fallback, in every block
            E = _push_below_zero(m, J, L, np.arange(5 + call, n, 11))
            ctx.set_radiation(J, L, E)
        ctx.get_populations_dev(d_old.data_ptr())
        before = ctx.get_populations()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ch_na, nf_na, rc_na = ctx.update_populations_noalloc(d_old.data_ptr(), d_new.data_ptr())
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (call, free0 - free1)   # no allocation, the first call included
        # the variant leaves the context's populations alone
        assert np.array_equal(ctx.get_populations(), before)
        got = d_new.cpu().numpy()
        ref, nf = o.stateq(J, L, E)
        _close_to_oracle(got, ref, m.n_spec)
        assert nf_na == nf and (nf > 0) == fallback
        assert abs(ch_na - o.max_rel_change(before, ref)) <= 1e-10 * ch_na
        ch, rc = ctx.update_populations()      # the existing entry point advances the context
        assert np.max(rel_err(got, ctx.get_populations())) < 1e-10
        assert abs(ch_na - ch) <= 1e-10 * ch
        assert rc_na == rc
        if fallback:
            assert rc == MG_WARN_NEG_POP_FALLBACK


def test_noalloc_refuses_bad_calls():
    import torch
    m = syn.model_sphere_1d(n=40, seed=1)
    ctx = gpu_context(m)
    ctx.trace_rays()
    ctx.init_populations()
    d = torch.empty((m.n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MagritteError) as e:   # no radiation field yet
        ctx.update_populations_noalloc(d.data_ptr(), d.data_ptr())
    assert e.value.code == MG_ERR_STATE
    ctx.formal_solve()
    with pytest.raises(mg.MagritteError) as e:
        ctx.update_populations_noalloc(0, d.data_ptr())
    assert e.value.code == MG_ERR_ARG


def test_noalloc_capacity_limit():
    """One cell beyond the static scratch's 2,097,152 gives MG_ERR_CAPACITY before any
    launch (a chain of points, 2-level species, radiation field set directly)."""
    import torch
    n = 2_097_153
    x = np.arange(n, dtype=np.float64) * 1e9
    pos = np.zeros((n, 3)); pos[:, 2] = x
    off = np.zeros(n + 1, np.int64); off[1:] = np.arange(1, n + 1)
    nbr = np.arange(1, n + 1, dtype=np.int32)
    nbr[-1] = n - 2
    bdy = np.zeros(n, np.uint8); bdy[-1] = 1
    sp = syn.species_two_level()
    ctx = mg.Context()
    ctx.set_mesh(pos, np.zeros((n, 3)), off, nbr, bdy)
    ctx.set_species(sp.E, sp.g, sp.mass, sp.up, sp.lo, sp.A, sp.T_grid, sp.K_down)
    one = np.ones(n)
    ctx.set_model(1e9 * one, 20.0 * one, 150.0 * one, 10.0 * one)
    ctx.init_populations()
    J = np.full((n, 1), 1e-17)
    ctx.set_radiation(J, np.zeros((n, 1)), J)
    d = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MagritteError) as e:
        ctx.update_populations_noalloc(d.data_ptr(), d.data_ptr())
    assert e.value.code == MG_ERR_CAPACITY
    ch, rc = ctx.update_populations()      # the regular update has no such limit
    assert np.isfinite(ch)
