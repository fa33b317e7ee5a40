"""Failure detection, determinism and checkpoint/resume of the CUDA path (no GPU fault is
ever provoked: failures are made on the host side, as bad inputs or call orders)."""
import numpy as np
import pytest

import synthetic as syn
from helpers import gpu_context, rel_err

pytestmark = pytest.mark.gpu


def _ready(prec=1, **kw):
    m = syn.model_clumpy_3d(n=1500, seed=31)
    ctx = gpu_context(m, precision=prec, **kw)
    ctx.trace_rays()
    ctx.init_populations()
    return m, ctx


@pytest.mark.parametrize("prec", [0, 1])
def test_reruns_are_bitwise_identical(prec):
    """Fixed-order reductions everywhere: two formal solves and two updates from the same
    populations give identical bits."""
    m, ctx = _ready(prec)
    outs = []
    for _ in range(2):
        ctx.init_populations()
        ctx.formal_solve()
        J, L, E = ctx.get_radiation()
        ch, _ = ctx.update_populations()
        outs.append((J, L, E, ctx.get_populations(), ch))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_not_converged_status_keeps_populations():
    import paper_1912_08445_gb300 as mg
    m, ctx = _ready(1, tol=1e-12, max_iter=2, ng_period=0)
    rep, rc = ctx.iterate(allow_not_converged=True)
    assert rc == mg.MG_ERR_NOT_CONVERGED and rep["iterations"] == 2 and not rep["converged"]
    assert np.all(np.isfinite(ctx.get_populations()))


def test_call_order_and_bad_inputs_are_rejected():
    import paper_1912_08445_gb300 as mg
    m = syn.model_tiny_3d(seed=2, n=12)
    ctx = mg.Context()
    with pytest.raises(mg.MagritteError) as e:
        ctx.formal_solve()
    assert e.value.code == mg.binding.MG_ERR_STATE
    bad = m.nbr_idx.copy(); bad[0] = m.n + 5                  # neighbour index out of range
    with pytest.raises(mg.MagritteError) as e:
        ctx.set_mesh(m.pos, m.vel, m.nbr_off, bad, m.is_bdy)
    assert e.value.code == mg.binding.MG_ERR_ARG
    ctx.set_mesh(m.pos, m.vel, m.nbr_off, m.nbr_idx, m.is_bdy)
    with pytest.raises(mg.MagritteError):
        ctx.set_model(m.n_coll, -m.T, m.v_turb, m.n_spec)      # negative temperature
    with pytest.raises(mg.MagritteError):
        ctx.trace_rays()                                       # no model, species, directions yet
    with pytest.raises(mg.MagritteError):
        ctx.set_quadrature(0)


def test_nonfinite_populations_fall_back_or_report():
    """Corrupt input populations (NaN in one cell): the statistical equilibrium repairs
    the cell through its fallback or reports MG_ERR_NUMERIC; it never returns silently
    non-finite populations."""
    import paper_1912_08445_gb300 as mg
    m, ctx = _ready(0)
    p = ctx.get_populations()
    p[7, :] = np.nan
    ctx.set_populations(p)
    ctx.formal_solve()
    try:
        ch, rc = ctx.update_populations()
    except mg.MagritteError as e:
        assert e.code == mg.binding.MG_ERR_NUMERIC
        return
    assert np.all(np.isfinite(np.delete(ctx.get_populations(), 7, axis=0)))


def test_checkpoint_resume_matches_uninterrupted_run():
    """Populations are the checkpoint: stopping after k iterations, restoring them into a
    fresh context and continuing gives the uninterrupted result."""
    m, ctx = _ready(1, tol=1e-300, max_iter=6, ng_period=0)
    ctx.iterate(allow_not_converged=True)
    full = ctx.get_populations()
    m2, c2 = _ready(1, tol=1e-300, max_iter=3, ng_period=0)
    c2.iterate(allow_not_converged=True)
    chk = c2.get_populations()
    m3, c3 = _ready(1, tol=1e-300, max_iter=3, ng_period=0)
    c3.set_populations(chk)
    c3.iterate(allow_not_converged=True)
    assert np.array_equal(c3.get_populations(), full)


def test_half_ray_beyond_max_steps_is_refused():
    """A half-ray longer than opt.max_steps cells ends the trace with MG_ERR_CAPACITY
    (nothing is stored); the same model traces with the default limit."""
    import paper_1912_08445_gb300 as mg
    m = syn.model_clumpy_3d(n=600, seed=4)
    ctx = gpu_context(m, max_steps=3)
    with pytest.raises(mg.MagritteError) as e:
        ctx.trace_rays()
    assert e.value.code == mg.binding.MG_ERR_CAPACITY
    with pytest.raises(mg.MagritteError) as e:
        ctx.formal_solve()
    assert e.value.code == mg.binding.MG_ERR_STATE
    ok = gpu_context(m)
    st, rc = ok.trace_rays()
    assert rc >= 0 and st["n_elements"] > 0
