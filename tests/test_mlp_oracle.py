"""Pins of the FP64 network oracle: finite-difference gradients, log-softmax identities,
Adam on a quadratic, and closed forms of the features."""
import numpy as np

import synthetic as syn
from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_out = 5
    theta = mlp.init_params(n_out, 1) * 0.5 + rng.normal(size=mlp.n_params(n_out)) * 0.01
    X = rng.normal(size=(7, 4))
    Y = rng.dirichlet(np.ones(n_out), size=7)
    Y[0, 2] = 1e-15      # masked entry
    L, g = mlp.loss_and_grad(theta, X, Y, n_out)
    idx = rng.choice(theta.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta); e[i] = 1e-6
        num = (mlp.loss(mlp.forward(theta + e, X, n_out)[0], Y) - mlp.loss(mlp.forward(theta - e, X, n_out)[0], Y)) / 2e-6
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, num, g[i])


def test_log_softmax_identities():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(6, 2)
    X = rng.normal(size=(11, 4))
    logp, _ = mlp.forward(theta, X, 6)
    assert np.allclose(np.exp(logp).sum(1), 1.0, atol=1e-14)
    # shifting the output bias by a constant leaves log p unchanged
    th2 = theta.copy(); th2[-6:] += 3.7
    assert np.allclose(mlp.forward(th2, X, 6)[0], logp, atol=1e-12)
    # loss is zero at the network's own output
    assert mlp.loss(logp, np.exp(logp)) < 1e-28


def test_adam_minimises_quadratic():
    theta = np.array([3.0, -2.0])
    m = np.zeros(2); v = np.zeros(2)
    for t in range(1, 2001):
        theta, m, v = mlp.adam_step(theta, 2 * theta, m, v, t, lr=0.05)
    assert np.abs(theta).max() < 1e-3


def test_features_closed_forms():
    """A uniform velocity gradient v = A x gives |grad v| = ||A||_F exactly (the
    least-squares fit is exact up to the 1e-6 regularisation); LTE Sobolev tau scales
    linearly with the species density."""
    m = syn.model_lattice_3d(m=5)
    A = np.array([[1e-9, 2e-9, 0], [0, -3e-9, 1e-9], [0.5e-9, 0, 2e-9]])
    m.vel = m.pos @ A.T
    m.T[:] = 30.0
    f = mlp.features(m)
    assert np.allclose(10 ** f[:, 2], np.sqrt((A * A).sum()), rtol=1e-5)
    assert np.allclose(f[:, 0], np.log10(m.n_coll)) and np.allclose(f[:, 1], np.log10(30.0))
    m2 = syn.model_lattice_3d(m=5)
    m2.vel = m.vel; m2.T[:] = 30.0; m2.n_spec = m.n_spec * 10
    f2 = mlp.features(m2)
    assert np.allclose(f2[:, 3] - f[:, 3], 1.0, atol=1e-12)
