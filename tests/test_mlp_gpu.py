"""Learned initial populations: the network kernels (BF16 tensor-core products, FP32
accumulation) against the FP64 network oracle, and the features against the oracle's."""
import numpy as np
import pytest

import synthetic as syn
from oracle import mlp as omlp
from helpers import gpu_context

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round-to-nearest-even to bfloat16, returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def bf16_forward(theta, X, n_out, mean, std):
    """The oracle's forward pass with the GPU's roundings: BF16 weights of the 128-wide
    layers and BF16 activations, FP64 arithmetic otherwise."""
    W1, b1, W2, b2, W3, b3, W4, b4 = omlp.unpack(theta.astype(np.float64), n_out)
    x = (X - mean) / std
    h1 = bf16(np.maximum(x @ W1 + b1, 0)).astype(np.float64)
    h2 = bf16(np.maximum(h1 @ bf16(W2) + b2, 0)).astype(np.float64)
    h3 = bf16(np.maximum(h2 @ bf16(W3) + b3, 0)).astype(np.float64)
    z = h3 @ bf16(W4) + b4
    z = z - z.max(1, keepdims=True)
    return z - np.log(np.exp(z).sum(1, keepdims=True))


def test_features_match_oracle():
    m = syn.model_clumpy_3d(n=2000, seed=21)
    ctx = gpu_context(m)
    f = ctx.features()
    fo = omlp.features(m)
    assert np.max(np.abs(f - fo)) < 2e-5


@pytest.mark.parametrize("n_out", [5, 20])
def test_forward_matches_oracle(n_out):
    import paper_1912_08445_gb300 as mg
    rng = np.random.default_rng(n_out)
    net = mg.MLP(n_out, seed=3)
    theta = omlp.init_params(n_out, 7).astype(np.float32)
    theta[-n_out:] = rng.normal(size=n_out)
    net.set_params(theta)
    mean = np.array([10.0, 1.5, -12.0, 0.0], np.float32); std = np.array([1.0, 0.3, 1.0, 2.0], np.float32)
    net.set_normalisation(mean, std)
    X = (mean + std * rng.normal(size=(1000, 4))).astype(np.float32)
    lp = net.forward(X)
    ref = bf16_forward(theta, X.astype(np.float64), n_out, mean, std)
    assert np.allclose(np.exp(lp).sum(1), 1.0, atol=1e-5)
    assert np.max(np.abs(lp - ref)) < 2e-2


@pytest.mark.parametrize("n_out", [5, 20])
def test_gradient_matches_oracle(n_out):
    """BF16 gradients against the FP64 backpropagation: cosine > 0.999 and relative
    norm error < 5e-2 for every parameter block."""
    import paper_1912_08445_gb300 as mg
    rng = np.random.default_rng(100 + n_out)
    net = mg.MLP(n_out, seed=3)
    theta = omlp.init_params(n_out, 9).astype(np.float32)
    net.set_params(theta)
    net.set_normalisation(np.zeros(4, np.float32), np.ones(4, np.float32))
    X = rng.normal(size=(700, 4)).astype(np.float32)
    Y = rng.dirichlet(np.ones(n_out) * 0.5, size=700).astype(np.float32)
    Y[Y < 1e-6] = 0.0
    loss, g = net.loss_grad(X, Y)
    L, go = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), n_out)
    assert abs(loss - L) < 2e-2 * L
    k = 0
    for s in omlp.shapes(n_out):
        m = int(np.prod(s))
        a, b = g[k:k + m].astype(np.float64), go[k:k + m]
        k += m
        if np.linalg.norm(b) < 1e-12:
            continue
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 0.999, (s, cos)
        assert np.linalg.norm(a - b) < 5e-2 * np.linalg.norm(b), s


def test_training_reduces_loss():
    """Fitting the outputs of a random teacher network: Adam on the GPU lowers the loss
    by more than an order of magnitude."""
    import paper_1912_08445_gb300 as mg
    n_out = 8
    rng = np.random.default_rng(5)
    teacher = omlp.init_params(n_out, 11)
    X = rng.normal(size=(20000, 4))
    Y = np.exp(omlp.forward(teacher, X, n_out)[0]).astype(np.float32)
    net = mg.MLP(n_out, seed=1)
    net.set_normalisation(np.zeros(4, np.float32), np.ones(4, np.float32))
    rep = net.train(X.astype(np.float32), Y, epochs=25, batch=1024, lr=2e-3, seed=0)
    assert rep["last_loss"] < rep["first_loss"] / 10, rep
    # the GPU loss agrees with the oracle's loss of the trained parameters
    th = net.get_params()
    lp = bf16_forward(th, X[:2000], n_out, np.zeros(4), np.ones(4))
    assert omlp.loss(lp, Y[:2000].astype(np.float64)) < rep["first_loss"] / 10


def test_save_load_attach(tmp_path):
    """A network written to a file and read back has the same parameters,
    normalisation and outputs; attached to a context it gives mg_init_populations
    (MG_INIT_MLP) the populations of mg_init_populations_mlp."""
    import paper_1912_08445_gb300 as mg
    m = syn.model_clumpy_3d(n=1500, seed=22)
    ctx = gpu_context(m)
    net = mg.MLP(ctx.n_lev, seed=5)
    net.set_normalisation([1.0, 2.0, -3.0, 0.5], [2.0, 0.5, 1.5, 3.0])
    path = tmp_path / "net.bin"
    net.save(path)
    back = mg.MLP.load(path)
    assert back.n_out == net.n_out and back.n_params == net.n_params
    assert np.array_equal(back.get_params(), net.get_params())
    X = np.random.default_rng(1).normal(size=(300, 4)).astype(np.float32)
    assert np.array_equal(back.forward(X), net.forward(X))
    # attached network: the init mode and the direct call agree bit for bit
    ctx.init_populations_mlp(back)
    direct = ctx.get_populations()
    ctx.init_populations()
    with pytest.raises(mg.MagritteError):
        ctx.init_populations(mg.MG_INIT_MLP)          # nothing attached yet
    ctx.attach_mlp(back)
    ctx.init_populations(mg.MG_INIT_MLP)
    assert np.array_equal(ctx.get_populations(), direct)
    # a file that is not a network is refused
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network file")
    with pytest.raises(mg.MagritteError):
        mg.MLP.load(bad)
    with pytest.raises(mg.MagritteError):
        ctx.attach_mlp(mg.MLP(ctx.n_lev + 1))      # outputs != levels
