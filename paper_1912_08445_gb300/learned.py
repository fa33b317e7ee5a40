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
