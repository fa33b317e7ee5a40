"""What the learned initial populations gain: trained on populations the ALI converged
to for seeded models, the network's start reaches the same fixed point in fewer
iterations than the LTE start on held-out seeds, and most where the ALI from LTE is
slow (discs with lines of optical depth ~1-10 and sub-thermal excitation)."""
import numpy as np
import pytest

import synthetic as syn
from helpers import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_1912_08445_gb300 import learned
    sp = syn.species_rotor(20, np.random.default_rng(77))
    train = learned.corpus_models(40, 1000, n_points=1500, species=sp, abundance_range=(1e-7, 1e-4))
    X, Y, reps = learned.build_corpus(train, ng_period=0)
    assert sum(r["converged"] for r in reps) >= 36
    net, trep = learned.train_network(X, Y, 20, epochs=40, batch=2048, lr=2e-3)
    assert trep["last_loss"] < trep["first_loss"]
    return sp, net


def _iterations(models, net):
    import paper_1912_08445_gb300 as mg
    it_lte, it_mlp = [], []
    for m in models:
        runs = {}
        for start in ("lte", "mlp"):
            ctx = mg.Context(precision=1, tol=1e-6, max_iter=400, ng_period=0)
            ctx.load_model(m)
            ctx.trace_rays()
            if start == "lte":
                ctx.init_populations()
            else:
                ctx.init_populations_mlp(net)
            rep, rc = ctx.iterate()
            runs[start] = (rep["iterations"], ctx.get_populations())
            ctx.close()
        it_lte.append(runs["lte"][0])
        it_mlp.append(runs["mlp"][0])
        # same fixed point from either start (the mixed path's tolerance)
        assert np.max(rel_err(runs["lte"][1], runs["mlp"][1])) < 1e-4
    return np.array(it_lte), np.array(it_mlp)


def test_learned_start_beats_lte_start(trained):
    from paper_1912_08445_gb300 import learned
    sp, net = trained
    held = learned.corpus_models(4, 5000, n_points=1500, species=sp, abundance_range=(1e-7, 1e-4))
    it_lte, it_mlp = _iterations(held, net)
    assert np.mean(it_mlp) < np.mean(it_lte), (it_lte, it_mlp)


def test_learned_start_on_slow_discs(trained):
    """Held-out discs where the ALI from LTE takes ~20 iterations: the network's start
    reaches the same fixed point, and in fewer iterations over the set (the gain is a few
    iterations: the error of either start falls by a constant factor per iteration, and
    the network's start is a few times closer than LTE, not orders of magnitude)."""
    from paper_1912_08445_gb300 import learned
    sp, net = trained
    slow = learned.slow_discs((5101,), n_points=1500, species=sp)
    it_lte, it_mlp = _iterations(slow, net)
    assert np.all(it_lte >= 15), it_lte
    assert np.all(it_mlp <= it_lte), (it_lte, it_mlp)
    assert np.sum(it_mlp) < np.sum(it_lte), (it_lte, it_mlp)
