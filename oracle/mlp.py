"""FP64 reference of the learned initial-population network (TEST INFRASTRUCTURE ONLY).

The network maps four local features of a cell to its fractional level populations:
  inputs  f = (log10 n_coll, log10 T, log10 |grad v|, log10 tau_Sobolev), normalised
          by a mean and standard deviation fixed at training time;
  hidden  three layers of 128 units with ReLU;
  output  n_lev logits -> log-softmax -> log fractional populations.
Loss: mean over (cell, level) pairs whose target fraction is >= 1e-12 of
(log p - log y)^2. Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
Parameters are one flat float vector: W1 [4][128], b1, W2 [128][128], b2, W3, b3,
W4 [128][n_out], b4 (weights stored [in][out]).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
N_IN = 4
FRAC_MIN = 1e-12
C_LIGHT = 299792458.0
H_PLANCK = 6.62607015e-34
K_BOLTZ = 1.380649e-23


def shapes(n_out):
    return [(N_IN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,),
            (HIDDEN, n_out), (n_out,)]


def n_params(n_out):
    return int(sum(np.prod(s) for s in shapes(n_out)))


def unpack(theta, n_out):
    out, k = [], 0
    for s in shapes(n_out):
        m = int(np.prod(s))
        out.append(theta[k:k + m].reshape(s))
        k += m
    return out


def init_params(n_out, seed):
    """He-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(n_out):
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[0])
            parts.append(rng.uniform(-lim, lim, s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def forward(theta, X, n_out):
    """Returns (log p [B][n_out], cache)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(np.asarray(theta, np.float64), n_out)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    a3 = h2 @ W3 + b3
    h3 = np.maximum(a3, 0.0)
    z = h3 @ W4 + b4
    zm = z - z.max(axis=1, keepdims=True)
    logp = zm - np.log(np.exp(zm).sum(axis=1, keepdims=True))
    return logp, (X, a1, h1, a2, h2, a3, h3, logp)


def loss(logp, Y):
    """Masked mean squared error of log fractions; Y holds target fractions."""
    mask = Y >= FRAC_MIN
    d = np.where(mask, logp - np.log(np.maximum(Y, FRAC_MIN)), 0.0)
    return float((d * d).sum() / max(int(mask.sum()), 1))


def loss_and_grad(theta, X, Y, n_out):
    """Loss and its gradient with respect to the flat parameters (backpropagation)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(np.asarray(theta, np.float64), n_out)
    logp, (X, a1, h1, a2, h2, a3, h3, _) = forward(theta, X, n_out)
    mask = Y >= FRAC_MIN
    cnt = max(int(mask.sum()), 1)
    d = np.where(mask, logp - np.log(np.maximum(Y, FRAC_MIN)), 0.0)
    L = float((d * d).sum() / cnt)
    g = 2.0 * d / cnt                           # dL/dlogp
    p = np.exp(logp)
    dz = g - p * g.sum(axis=1, keepdims=True)   # through log-softmax
    dW4 = h3.T @ dz
    db4 = dz.sum(0)
    dh3 = (dz @ W4.T) * (a3 > 0)
    dW3 = h2.T @ dh3
    db3 = dh3.sum(0)
    dh2 = (dh3 @ W3.T) * (a2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    dW1 = X.T @ dh1
    db1 = dh1.sum(0)
    grad = np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3, dW4, db4)])
    return L, grad


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(model):
    """Per-cell network inputs (before normalisation), FP64:
      log10 n_coll, log10 T,
      log10 |grad v|: Frobenius norm of the least-squares velocity gradient G over the
        neighbour list, G = (sum dv dx^T)(sum dx dx^T + 1e-6 tr/3 I)^-1 (floor 1e-30),
      log10 tau: Sobolev optical depth of line 0 at LTE populations,
        chi_int c / (nu max(|grad v|, b / l)), with l the mean neighbour distance and b
        the local velocity width (floor 1e-30)."""
    m = model
    sp = m.species
    n = m.n
    out = np.zeros((n, 4))
    nu = (sp.E[sp.up[0]] - sp.E[sp.lo[0]]) / H_PLANCK
    Bul = sp.A[0] * C_LIGHT ** 2 / (2 * H_PLANCK * nu ** 3)
    Blu = sp.g[sp.up[0]] / sp.g[sp.lo[0]] * Bul
    for c in range(n):
        nb = m.nbr_idx[m.nbr_off[c]:m.nbr_off[c + 1]]
        dx = m.pos[nb] - m.pos[c]
        dv = m.vel[nb] - m.vel[c]
        M = dx.T @ dx
        M = M + 1e-6 * np.trace(M) / 3.0 * np.eye(3)
        Bm = dv.T @ dx
        G = Bm @ np.linalg.inv(M) if len(nb) else np.zeros((3, 3))
        gv = float(np.sqrt((G * G).sum()))
        ell = float(np.linalg.norm(dx, axis=1).mean()) if len(nb) else 1.0
        b = np.sqrt(2 * K_BOLTZ * m.T[c] / sp.mass + m.v_turb[c] ** 2)
        Z = (sp.g * np.exp(-sp.E / (K_BOLTZ * m.T[c]))).sum()
        nl = m.n_spec[c] * sp.g[sp.lo[0]] * np.exp(-sp.E[sp.lo[0]] / (K_BOLTZ * m.T[c])) / Z
        nu_ = m.n_spec[c] * sp.g[sp.up[0]] * np.exp(-sp.E[sp.up[0]] / (K_BOLTZ * m.T[c])) / Z
        chi_int = H_PLANCK * nu / (4 * np.pi) * (nl * Blu - nu_ * Bul)
        tau = chi_int * C_LIGHT / (nu * max(gv, b / ell))
        out[c] = (np.log10(m.n_coll[c]), np.log10(m.T[c]), np.log10(max(gv, 1e-30)), np.log10(max(tau, 1e-30)))
    return out
