"""Batched models (uneven sizes, one persistent launch per iteration, CUDA graphs):
identical to solving each model on its own, and within the mixed tolerance of the
oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle
from helpers import rel_err, gpu_context

pytestmark = pytest.mark.gpu


def _models(k=6, seed=11, n_q=31):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(600), np.log(4000), k)).astype(int)
    return [syn.model_clumpy_3d(n=int(s), seed=seed * 100 + i, v_max=float(rng.uniform(2e3, 2e4)), n_q=n_q)
            for i, s in enumerate(sizes)]


def test_batch_formal_solve_matches_single_models():
    import paper_1912_08445_gb300 as mg
    ms = _models()
    ctxs = []
    for m in ms:
        c = gpu_context(m, precision=1)
        c.trace_rays()
        c.init_populations()
        ctxs.append(c)
    refs = []
    for c in ctxs:
        c.formal_solve()
        refs.append(c.get_radiation())
    b = mg.Batch(ctxs)
    b.formal_solve()
    for c, (J, L, E) in zip(ctxs, refs):
        J2, L2, E2 = c.get_radiation()
        assert np.max(rel_err(J2, J)) < 1e-12
        assert np.max(rel_err(E2, E)) < 1e-12
        assert np.max(np.abs(L2 - L)) < 1e-12
    v, srt, ms_ = b.autotune(reps=1)
    assert v >= 0
    # every model still within the mixed tolerance of the oracle after autotuning
    o = Oracle(ms[1], nthreads=16)
    origins = np.sort(np.random.default_rng(0).choice(ms[1].n, 20, replace=False))
    Jo, Lo, Eo = o.formal_solve(o.lte(), origins)
    J2, L2, E2 = ctxs[1].get_radiation()
    assert np.max(rel_err(J2[origins], Jo)) < 1e-4
    b.close()


@pytest.mark.parametrize("ng", [0, 4])
def test_batch_ali_matches_single_model_ali(ng):
    """The batched ALI takes the same iterations (and, with Ng, the same Ng steps) as
    each model's own mg_iterate and reaches the same populations."""
    import paper_1912_08445_gb300 as mg
    ms = _models(k=5, seed=12)
    singles, batched = [], []
    for m in ms:
        c = gpu_context(m, precision=1, tol=1e-6, max_iter=100, ng_period=ng)
        c.trace_rays()
        c.init_populations()
        rep, rc = c.iterate()
        singles.append((rep, c.get_populations()))
    ctxs = []
    for m in ms:
        c = gpu_context(m, precision=1, tol=1e-6, max_iter=100, ng_period=ng)
        c.trace_rays()
        c.init_populations()
        ctxs.append(c)
    b = mg.Batch(ctxs)
    reps, rc = b.iterate()
    assert rc == 0
    for (rep, pops), r2, c in zip(singles, reps, ctxs):
        assert r2["converged"] and r2["iterations"] == rep["iterations"]
        assert r2["ng_steps"] == rep["ng_steps"]
        assert np.max(rel_err(c.get_populations(), pops)) < 1e-12
    b.close()


@pytest.mark.parametrize("Q,variants", [(31, [0, 1, 2, 3, 4, 11, 12, 13, 14, 15, 16, 17, 24, 25]),
                                        (63, [10, 23, 28, 29, 30, 31])])
def test_every_batch_variant_does_the_work(Q, variants):
    """Every launch variant valid for 4 lines x Q bins, in both queue orders, gives the
    persistent batch kernel the same radiation field as the per-model launch of that
    variant (the batch holds a work-item list for every lines-per-warp value; variants
    28-31 run three warps per block)."""
    import paper_1912_08445_gb300 as mg
    ms = _models(k=3, seed=5, n_q=Q)
    ctxs = []
    for m in ms:
        c = gpu_context(m, precision=1)
        c.trace_rays()
        c.init_populations()
        ctxs.append(c)
    b = mg.Batch(ctxs)
    for v in variants:
        refs = []
        for c in ctxs:
            c.set_variant(v)
            c.formal_solve()
            refs.append(c.get_radiation())
        for srt in (True, False):
            # leave another field (every molecule in the ground level) in the buffers, so
            # that a launch doing nothing is caught, then restore the populations
            for c in ctxs:
                p1 = c.get_populations()
                p2 = np.zeros_like(p1)
                p2[:, 0] = p1.sum(axis=1)
                c.set_populations(p2)
                c.formal_solve()
                c.set_populations(p1)
            b.set_variant(v, srt)
            b.formal_solve()
            for c, (J, L, E) in zip(ctxs, refs):
                J2, L2, E2 = c.get_radiation()
                assert np.max(rel_err(J2, J)) < 1e-12, (v, srt)
                assert np.max(rel_err(E2, E)) < 1e-12, (v, srt)
    with pytest.raises(mg.MagritteError):
        b.set_variant(5 if Q == 31 else 0)   # not valid for Q bins
    b.close()
