"""Learned initial populations: corpus of converged ALI solutions -> trained network ->
initial populations for new models. Orchestration only: every step runs in the library's
kernels (ALI, features, training, inference)."""
from __future__ import annotations

import numpy as np

from .binding import Context, MLP, MG_MIXED


def converged_rows(model, tol=1e-6, max_iter=300, ng_period=4, precision=MG_MIXED):
    """Features [n][4] and converged fractional populations [n][n_lev] of one model,
    plus the ALI report from an LTE start."""
    ctx = Context(precision=precision, tol=tol, max_iter=max_iter, ng_period=ng_period)
    ctx.load_model(model)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate(allow_not_converged=True)
    pops = ctx.get_populations()
    feats = ctx.features()
    ctx.close()
    return feats, (pops / model.n_spec[:, None]).astype(np.float32), rep


def build_corpus(models, **kw):
    X, Y, reps = [], [], []
    for m in models:
        f, y, rep = converged_rows(m, **kw)
        if rep["converged"]:
            X.append(f); Y.append(y)
        reps.append(rep)
    return np.concatenate(X), np.concatenate(Y), reps


def train_network(X, Y, n_lev, epochs=30, batch=4096, lr=2e-3, seed=0, device=0):
    """Trains a network on (features, fractions); inputs normalised by their corpus mean
    and standard deviation."""
    net = MLP(n_lev, seed=seed, device=device)
    mean = X.mean(0)
    std = np.maximum(X.std(0), 1e-3)
    net.set_normalisation(mean, std)
    rep = net.train(X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, rep


def corpus_models(n_models, seed0, n_points=3000, species=None, abundance_range=(1e-7, 1e-5)):
    """Seeded cloud/disc models of the given species (alternating shapes of the clumpy
    cloud and the Keplerian disc, scaled down), densities and abundances log-uniform."""
    import synthetic as syn
    out = []
    for k in range(n_models):
        rng = np.random.default_rng(seed0 + k)
        dens = float(np.exp(rng.uniform(np.log(1e8), np.log(1e11))))
        X = float(np.exp(rng.uniform(np.log(abundance_range[0]), np.log(abundance_range[1]))))
        if k % 2 == 0:
            m = syn.model_clumpy_3d(n=n_points, seed=seed0 + k, n_h2_ref=dens, abundance=X, species=species,
                                    v_max=float(rng.uniform(2e3, 2e4)))
        else:
            m = syn.model_disc(n=n_points, seed=seed0 + k, nside=2, n_q=31, n_lev=species.n_lev,
                               n_h2_in=dens * 100, abundance=X)
            m.species = species
        out.append(m)
    return out


def slow_discs(seeds, n_points=3000, species=None, densities=(1e12, 3e12, 1e13), abundance=1e-4):
    """Held-out discs in the regime where the ALI from LTE is slow (lines of optical depth
    ~1-10 with sub-thermal excitation: 19-21 iterations from LTE at 3000 points)."""
    import synthetic as syn
    out = []
    for s in seeds:
        for d in densities:
            m = syn.model_disc(n=n_points, seed=s, nside=2, n_q=31, n_lev=species.n_lev, n_h2_in=d,
                               abundance=abundance)
            m.species = species
            out.append(m)
    return out
