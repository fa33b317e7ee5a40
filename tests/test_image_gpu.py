"""Images (Sec. 3.5, 'Imaging the model') through the CUDA library against the oracle:
intensity per point and channel within 1e-10 relative in FP64 contexts and 1e-4 in
mixed-precision contexts (FP32 image kernel), sky-plane coordinates within 1e-12."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle
from helpers import rel_err, gpu_context
import paper_1912_08445_gb300 as mg
from paper_1912_08445_gb300.binding import MG_ERR_ARG, MG_ERR_STATE

pytestmark = pytest.mark.gpu
TOL = 1e-10
TOL_MIX = 1e-4


def _lattice_flow():
    m = syn.model_lattice_3d(m=9)
    m.vel = np.zeros_like(m.pos)
    m.vel[:, 2] = 1e4 / 8e12 * m.pos[:, 2]
    m.n_spec = np.full(m.n, 1e3)
    return m


CASES = {
    "tiny": (lambda: syn.model_tiny_3d(seed=4, n=20), None, [0, 3]),
    "lattice_flow": (_lattice_flow, None, [0, 5]),
    "hubble_line": (lambda: syn.hubble_line_1d(n_cells=100, n_q=31), None, [0, 1]),
    "sphere1d": (lambda: syn.vz_problem1(abundance=1e-6, v_inf=1e4, n_shells=50), None, [0, 13]),
    "clumpy3000": (lambda: syn.model_clumpy_3d(n=3000, seed=3), 150, [0, 21, 40]),
}


def _compare(m, o, ctx, rays, origins, pops=None, n_ch=41, tol=TOL):
    pops = o.lte() if pops is None else pops
    for r in rays:
        for line in range(m.species.n_lines):
            b = o.width(0)
            u = np.linspace(-10, 10, n_ch) * b
            I, xy = ctx.image(r, line, u)
            Io, xyo = o.image(pops, r, line, u, origins=origins)
            sel = slice(None) if origins is None else origins
            assert np.max(rel_err(I[sel], Io)) < tol, (r, line)
            scale = np.abs(m.pos).max()
            assert np.max(np.abs(xy[sel] - xyo)) <= 1e-12 * scale
            if line >= 1:
                break


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_image_matches_oracle(name, precision):
    make, n_orig, rays = CASES[name]
    m = make()
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=precision)
    ctx.trace_rays()
    ctx.init_populations()
    origins = None if n_orig is None else np.sort(np.random.default_rng(2).choice(m.n, n_orig, replace=False))
    _compare(m, o, ctx, rays, origins, tol=TOL if precision == 0 else TOL_MIX)


def test_image_uses_current_populations():
    """After an ALI (mixed precision) the image follows the iterated populations, not LTE."""
    m = syn.model_clumpy_3d(n=2000, seed=11)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, precision=1, tol=1e-6, max_iter=60, ng_period=4)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.iterate(allow_not_converged=True)
    pops = ctx.get_populations()
    origins = np.sort(np.random.default_rng(4).choice(m.n, 100, replace=False))
    _compare(m, o, ctx, [7], origins, pops=pops, tol=TOL_MIX)
    u = np.linspace(-10, 10, 41) * o.width(0)
    I_lte, _ = o.image(o.lte(), 7, 0, u, origins=origins)
    I, _ = ctx.image(7, 0, u)
    assert np.max(rel_err(I[origins], I_lte)) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_image_disc_200k_sampled(precision):
    """Full-size Keplerian disc (200k points, 192 rays, 20-level rotor): one image of the
    lowest line with 63 channels, checked against the oracle on 60 sampled points."""
    m = syn.model_disc()
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, precision=precision, profile=1)
    ctx.trace_rays()
    ctx.init_populations()
    origins = np.sort(np.random.default_rng(5).choice(m.n, 60, replace=False))
    u = np.linspace(-15e3, 15e3, 63)
    ray = 40
    I, xy = ctx.image(ray, 0, u)
    Io, xyo = o.image(o.lte(), ray, 0, u, origins=origins)
    assert np.max(rel_err(I[origins], Io)) < (TOL if precision == 0 else TOL_MIX)
    assert np.all(np.isfinite(I)) and np.all(I > 0)
    assert ("image_fp64" if precision == 0 else "image_fp32") in ctx.kernel_times()


def test_image_dev_equals_host():
    import torch
    m = syn.model_clumpy_3d(n=3000, seed=3)
    ctx = gpu_context(m, precision=1)
    ctx.trace_rays()
    ctx.init_populations()
    u = np.linspace(-5e3, 5e3, 17)
    I, xy = ctx.image(3, 1, u)
    dI = torch.empty((m.n, 17), dtype=torch.float64, device="cuda")
    dxy = torch.empty((m.n, 2), dtype=torch.float64, device="cuda")
    ctx.image_dev(3, 1, u, dI.data_ptr(), dxy.data_ptr())
    assert np.array_equal(dI.cpu().numpy(), I) and np.array_equal(dxy.cpu().numpy(), xy)


def test_image_bad_calls():
    m = syn.model_tiny_3d(seed=4, n=20)
    ctx = gpu_context(m)
    u = np.zeros(3)
    with pytest.raises(mg.MagritteError) as e:
        ctx.image(0, 0, u)
    assert e.value.code == MG_ERR_STATE
    ctx.trace_rays()
    ctx.init_populations()
    R = 12 * m.nside ** 2
    for ray, line, uu in ((-1, 0, u), (R, 0, u), (0, -1, u), (0, m.species.n_lines, u),
                          (0, 0, np.zeros(0)), (0, 0, np.array([np.nan])), (0, 0, np.array([1e8]))):
        with pytest.raises(mg.MagritteError) as e:
            ctx.image(ray, line, uu)
        assert e.value.code == MG_ERR_ARG
    I, xy = ctx.image(0, 0, u)
    assert np.all(np.isfinite(I))


def test_image_after_mesh_change():
    """A context reloaded with a larger mesh (and another species) images the new model:
    the image buffers follow the point and line counts."""
    import paper_1912_08445_gb300 as mgp
    small = syn.model_clumpy_3d(n=600, seed=8)
    big = syn.model_clumpy_3d(n=3000, seed=9, n_lev=7)
    ctx = mgp.Context(precision=1)
    u = np.linspace(-3e3, 3e3, 9)
    for m in (small, big):
        o = Oracle(m, nthreads=16)
        ctx.load_model(m, dirs=o.dirs)
        ctx.trace_rays()
        ctx.init_populations()
        I, xy = ctx.image(5, 1, u)
        assert I.shape == (m.n, 9)
        origins = np.arange(0, m.n, 37)
        Io, _ = o.image(o.lte(), 5, 1, u, origins=origins)
        assert np.max(rel_err(I[origins], Io)) < TOL_MIX
