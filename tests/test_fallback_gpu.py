"""Validity check of Sec. 6.1 on the GPU against the oracle: a cell whose ALO-corrected
rates give a negative population is solved again without the ALO (L = 0, J_eff = J) and
counted. The radiation field is given through mg_set_radiation, so that the statistical
equilibrium of mg_update_populations (FP64 in both precisions) meets exactly the rates
the oracle's pin uses."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle, CONST
from helpers import rel_err, gpu_context
from paper_1912_08445_gb300.binding import MG_WARN_NEG_POP_FALLBACK

pytestmark = pytest.mark.gpu
h, kB, c = CONST["h"], CONST["kB"], CONST["c"]


def _two_cell_model(n_coll, T=30.0):
    sp = syn.species_two_level(A21=1e-5)
    return syn.model_line_1d(np.array([0.0, 1e10]), 0.0, n_coll, T, 150.0, 1e-8, sp, 5)


def _negative_excitation(m, J, L, cells):
    """J_eff of the given cells of a 2-level model set so that the excitation rate
    B_lu J_eff + C_lu is -C_lu/2 < 0 while the de-excitation rate stays positive: the
    ALO solution of those cells has a negative upper population."""
    sp = m.species
    nu = (sp.E[1] - sp.E[0]) / h
    Bul = sp.A[0] * c ** 2 / (2 * h * nu ** 3)
    Blu = sp.g[1] / sp.g[0] * Bul
    E = J.copy()
    for cc in cells:
        Cd = float(sp.K_down[0, 0]) * m.n_coll[cc]
        Cu = Cd * sp.g[1] / sp.g[0] * math.exp(-h * nu / (kB * m.T[cc]))
        E[cc, 0] = -1.5 * Cu / Blu
        assert sp.A[0] * (1 - L[cc, 0]) + Bul * E[cc, 0] + Cd > 0
    return E


@pytest.mark.parametrize("precision", [0, 1])
def test_two_cell_fallback_matches_oracle(precision):
    """The oracle pin's case: cell 1 with J_eff = -0.03 J takes the fallback, cell 0 keeps
    its ALO solution; populations within 1e-10 of the oracle (the update is FP64 in both
    precisions), one fallback cell, status MG_WARN_NEG_POP_FALLBACK."""
    m = _two_cell_model(1e9)
    o = Oracle(m)
    ctx = gpu_context(m, precision=precision)
    ctx.init_populations()
    Jv, Lv = 1e-16, 0.9
    J = np.full((2, 1), Jv)
    L = np.full((2, 1), Lv)
    E = np.array([[0.5 * Jv], [-0.03 * Jv]])
    ctx.set_radiation(J, L, E)
    ch, rc = ctx.update_populations()
    ref, nf = o.stateq(J, L, E)
    assert nf == 1
    assert rc == MG_WARN_NEG_POP_FALLBACK
    assert ctx.status_counts()[0] == nf
    pops = ctx.get_populations()
    assert np.max(rel_err(pops, ref)) < 1e-10
    assert np.all(pops >= 0)


@pytest.mark.parametrize("precision", [0, 1])
def test_fallback_cells_of_a_solved_model_match_oracle(precision):
    """A 300-shell 1D cloud (three blocks of the update kernel): the radiation field of a
    formal solve, with J_eff of every 7th cell pushed below zero. Exactly those cells fall
    back; all populations within 1e-10 of the oracle's update of the same field."""
    m = syn.model_sphere_1d(n=300, seed=5)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=precision)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E0 = ctx.get_radiation()
    cells = np.arange(3, m.n, 7)
    E = _negative_excitation(m, J, L, cells)
    ctx.set_radiation(J, L, E)
    ch, rc = ctx.update_populations()
    ref, nf = o.stateq(J, L, E)
    assert nf == len(cells)
    assert rc == MG_WARN_NEG_POP_FALLBACK and ctx.status_counts()[0] == nf
    pops = ctx.get_populations()
    assert np.max(rel_err(pops, ref)) < 1e-10
    assert np.all(pops >= 0)
    assert abs(ch - o.max_rel_change(o.lte(), ref)) <= 1e-10 * ch
