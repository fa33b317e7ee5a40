"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs. Ray tracing is compared bit for bit; FP64 radiation fields and
populations within 1e-10 relative (the FP64 tolerance of the method's GPU path)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Oracle, healpix_dirs, gauss_hermite
from helpers import rel_err, gpu_context, compare_rays

pytestmark = pytest.mark.gpu
TOL64 = 1e-10


def small_clumpy(n=3000, seed=3):
    return syn.model_clumpy_3d(n=n, seed=seed)


# ------------------------------------------------------------------ set-up tables
@pytest.mark.parametrize("nside", [1, 2, 4])
def test_healpix_matches_oracle(nside):
    import paper_1912_08445_gb300 as mg
    ctx = mg.Context()
    ctx.set_directions(nside)
    d, a = ctx.get_directions()
    ref = healpix_dirs(nside)
    assert d.shape == ref.shape
    assert np.abs(d - ref).max() < 1e-15
    assert np.all(np.abs(d + d[a]).max(1) < 1e-15)


@pytest.mark.parametrize("Q", [1, 7, 31, 63, 100])
def test_quadrature_matches_oracle(Q):
    import paper_1912_08445_gb300 as mg
    ctx = mg.Context()
    ctx.set_quadrature(Q)
    r, w = ctx.get_quadrature()
    r0, w0 = gauss_hermite(Q)
    assert np.abs(r - r0).max() < 1e-12
    assert np.abs(w - w0).max() < 1e-13


# ------------------------------------------------------------------ ray tracing
def _moved(m, scale=1.0, shift=0.0):
    """The same cloud with its positions scaled and shifted (the walk's FP32 filter meets
    overflowing squares, or bounds too wide to decide, and must defer to FP64)."""
    import dataclasses
    return dataclasses.replace(m, pos=m.pos * scale + shift)


@pytest.mark.parametrize("name", ["tiny", "lattice", "sphere1d", "clumpy3000", "hubble_fast",
                                  "clumpy_huge_scale", "clumpy_far_offset"])
def test_trace_bit_exact(name):
    m = {"tiny": lambda: syn.model_tiny_3d(seed=4, n=20),
         "lattice": lambda: syn.model_lattice_3d(m=6),
         "sphere1d": lambda: syn.model_sphere_1d(n=200, seed=1),
         "clumpy3000": lambda: small_clumpy(),
         "hubble_fast": lambda: syn.hubble_line_1d(n_cells=60, c_dbeta=0.5),
         # squares of 1e35 m overflow FP32: every comparison goes to FP64
         "clumpy_huge_scale": lambda: _moved(small_clumpy(n=1500, seed=8), scale=1e22),
         # a cloud 1e6 radii from the origin of coordinates: FP32 positions resolve only
         # ~1/6 of a cell spacing, so many decisions are left to FP64
         "clumpy_far_offset": lambda: _moved(small_clumpy(n=1500, seed=9), shift=1e21)}[name]()
    o = Oracle(m, nthreads=8)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    st, rc = ctx.trace_rays()
    origins = np.arange(m.n)
    tr = o.trace_all(origins)
    assert st["n_elements"] == tr["off"][-1]
    assert st["n_expanded"] == tr["off"][-1] + tr["nsub"].sum()
    assert st["n_dead_end"] == tr["dead"].sum()
    bad = compare_rays(ctx, tr, origins, o.dirs.shape[0])
    assert not bad, bad[:10]


def test_trace_bit_exact_clumpy_50k():
    """Full-size 3D clumpy cloud (50k points, 48 rays): every half-ray bit-exact; the
    per-ray comparison samples 2000 origins, the totals cover all 2.4M half-rays."""
    m = syn.model_clumpy_3d(n=50_000, seed=0)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    st, _ = ctx.trace_rays()
    tr_all = o.trace_all()
    assert st["n_elements"] == tr_all["off"][-1]
    assert st["n_expanded"] == tr_all["off"][-1] + tr_all["nsub"].sum()
    assert st["n_dead_end"] == tr_all["dead"].sum()
    rng = np.random.default_rng(0)
    origins = np.sort(rng.choice(m.n, 2000, replace=False))
    tr = o.trace_all(origins)
    bad = compare_rays(ctx, tr, origins, o.dirs.shape[0])
    assert not bad, bad[:10]


# ------------------------------------------------------------------ formal solve (FP64)
def _fs_case(name):
    if name == "sphere1d":
        return syn.model_sphere_1d(n=200, seed=1), None
    if name == "sphere1d_thick":
        m = syn.model_sphere_1d(n=120, seed=2)
        m.n_spec = m.n_spec * 3e3
        return m, None
    if name == "tiny":
        return syn.model_tiny_3d(seed=4, n=20), None
    if name == "hubble":
        return syn.hubble_line_1d(n_cells=100, n_q=31), None
    if name == "powerlaw":
        m = syn.powerlaw_line_1d(n_shells=50, n_q=31)
        return m, None
    if name == "clumpy3000":
        return small_clumpy(), np.sort(np.random.default_rng(1).choice(3000, 150, replace=False))
    raise KeyError(name)


@pytest.mark.parametrize("name", ["sphere1d", "sphere1d_thick", "tiny", "hubble", "powerlaw", "clumpy3000"])
def test_formal_solve_fp64_parity(name):
    m, origins = _fs_case(name)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, spectrum=1)
    ctx.trace_rays()
    ctx.init_populations()
    pops = ctx.get_populations()
    ref_pops = o.lte()
    assert np.max(rel_err(pops, ref_pops)) < 1e-14
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    Jnu = ctx.get_spectrum()
    sel = slice(None) if origins is None else origins
    Jo, Lo, Eo, Jnuo = o.formal_solve(ref_pops, origins, spectrum=True)
    assert np.max(rel_err(J[sel], Jo)) < TOL64
    assert np.max(rel_err(E[sel], Eo)) < TOL64
    assert np.max(rel_err(L[sel], Lo, floor=1e-300)) < TOL64
    assert np.max(rel_err(Jnu[sel], Jnuo)) < TOL64


def test_formal_solve_fp64_clumpy_50k_sampled():
    """Full-size clumpy cloud (50k points, 48 rays, 4 lines x 31 bins) in FP64: sampled
    origins against the oracle."""
    m = syn.model_clumpy_3d(n=50_000, seed=0)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    origins = np.sort(np.random.default_rng(2).choice(m.n, 24, replace=False))
    Jo, Lo, Eo = o.formal_solve(o.lte(), origins)
    assert np.max(rel_err(J[origins], Jo)) < TOL64
    assert np.max(rel_err(E[origins], Eo)) < TOL64
    assert np.max(rel_err(L[origins], Lo, floor=1e-300)) < TOL64


# ------------------------------------------------------------------ statistical equilibrium and ALI
@pytest.mark.parametrize("name", ["sphere1d", "sphere1d_thick", "tiny"])
def test_one_iteration_parity(name):
    m, _ = _fs_case(name)
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    ctx.trace_rays()
    ctx.init_populations()
    ctx.formal_solve()
    ch, rc = ctx.update_populations()
    pops = ctx.get_populations()
    p0 = o.lte()
    J, L, E = o.formal_solve(p0)
    ref, nf = o.stateq(J, L, E)
    assert nf == 0 and rc == 0
    assert np.max(rel_err(pops, ref)) < TOL64
    assert abs(ch - o.max_rel_change(p0, ref)) <= 1e-9 * max(ch, 1e-300)


@pytest.mark.parametrize("ng", [0, 4])
def test_ali_iterations_parity(ng):
    """Same number of ALI iterations from the same LTE start: populations within 1e-10."""
    m, _ = _fs_case("sphere1d_thick")
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, tol=1e-300, max_iter=12, ng_period=ng)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate(allow_not_converged=True)
    assert rep["iterations"] == 12
    pops = ctx.get_populations()
    ref, ch, conv = o.ali(tol=1e-300, max_iter=12, ng_period=ng)
    assert len(ch) == 12
    tol = TOL64 if ng == 0 else 1e-8
    assert np.max(rel_err(pops, ref)) < tol


def test_ali_converges_to_oracle_fixed_point():
    m, _ = _fs_case("sphere1d_thick")
    o = Oracle(m, nthreads=16)
    ctx = gpu_context(m, oracle_dirs=o.dirs, tol=1e-12, max_iter=400, ng_period=4)
    ctx.trace_rays()
    ctx.init_populations()
    rep, rc = ctx.iterate()
    assert rep["converged"]
    ref, ch, conv = o.ali(tol=1e-12, max_iter=400, ng_period=0)
    assert conv
    assert np.max(rel_err(ctx.get_populations(), ref)) < 1e-9


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("precision", [0, 1])
def test_isolated_and_boundary_points(precision):
    """A point with no neighbours (both half-rays empty: u = I_cmb, Lambda* = 0) and
    boundary origins with outward rays that end immediately, in FP64 (1e-10) and in mixed
    precision (the warp kernel's empty-half and isolated-origin paths, 1e-4)."""
    m = syn.model_tiny_3d(seed=5, n=12)
    # cut every neighbour link of point 0
    keep = []
    off = [0]
    for i in range(m.n):
        row = [j for j in m.nbr_idx[m.nbr_off[i]:m.nbr_off[i + 1]] if j != 0 and i != 0]
        keep.extend(row)
        off.append(len(keep))
    m.nbr_idx = np.array(keep, np.int32)
    m.nbr_off = np.array(off, np.int64)
    o = Oracle(m, nthreads=4)
    ctx = gpu_context(m, oracle_dirs=o.dirs, spectrum=1, precision=precision)
    st, rc = ctx.trace_rays()
    assert rc == 1 and st["n_dead_end"] >= o.dirs.shape[0]
    ctx.init_populations()
    ctx.formal_solve()
    J, L, E = ctx.get_radiation()
    Jo, Lo, Eo = o.formal_solve(o.lte())
    tol = TOL64 if precision == 0 else 1e-4
    assert np.max(rel_err(J, Jo)) < tol
    assert np.max(rel_err(E, Eo)) < tol
    assert np.all(L[0] == 0.0)


def test_single_point_and_empty_models():
    """A one-point model (no neighbours at all: every half-ray empty) is solved like an
    isolated point; an empty mesh is refused with MG_ERR_ARG before anything runs."""
    import paper_1912_08445_gb300 as mg
    m = syn.model_tiny_3d(seed=5, n=12)
    one = syn.Model(name="one", pos=m.pos[:1].copy(), vel=m.vel[:1].copy(), nbr_off=np.zeros(2, np.int64),
                    nbr_idx=np.zeros(0, np.int32), is_bdy=np.ones(1, np.uint8), n_coll=m.n_coll[:1].copy(),
                    T=m.T[:1].copy(), v_turb=m.v_turb[:1].copy(), n_spec=m.n_spec[:1].copy(), species=m.species,
                    geometry=m.geometry, nside=m.nside, n_q=m.n_q)
    o = Oracle(one, nthreads=1)
    for precision in (0, 1):
        ctx = gpu_context(one, oracle_dirs=o.dirs, precision=precision)
        ctx.trace_rays()
        ctx.init_populations()
        ctx.formal_solve()
        J, L, E = ctx.get_radiation()
        Jo, Lo, Eo = o.formal_solve(o.lte())
        assert np.max(rel_err(J, Jo)) < (TOL64 if precision == 0 else 1e-4)
        assert np.all(L == 0.0)
        ctx.update_populations()
        assert np.all(np.isfinite(ctx.get_populations()))
    ctx = mg.Context()
    with pytest.raises(mg.MagritteError) as e:
        ctx.set_mesh(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(1, np.int64), np.zeros(0, np.int32),
                     np.zeros(0, np.uint8))
    assert e.value.code == mg.binding.MG_ERR_ARG


def test_negative_opacity_is_reported():
    """A population inversion (n_u/g_u > n_l/g_l: a maser, which the method does not
    treat) makes the line opacity integral negative: the update reports
    MG_WARN_NEG_OPACITY and counts the (point, line) pairs."""
    import paper_1912_08445_gb300 as mg
    m = syn.model_tiny_3d(seed=4, n=20)
    o = Oracle(m, nthreads=4)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    ctx.trace_rays()
    pops = o.lte()
    sp = m.species
    u, lo = int(sp.up[0]), int(sp.lo[0])
    pops[3, u] = pops[3, lo] * sp.g[u] / sp.g[lo] * 1.5     # invert line 0 in point 3
    ctx.set_populations(pops)
    ctx.formal_solve()
    ch, rc = ctx.update_populations()
    fb, neg = ctx.status_counts()
    assert neg == 1
    assert rc in (mg.MG_WARN_NEG_OPACITY, mg.MG_WARN_NEG_POP_FALLBACK)
    ctx.init_populations()
    ctx.formal_solve()
    ch, rc = ctx.update_populations()
    assert ctx.status_counts()[1] == 0 and rc == 0


def test_trace_tie_breaks_bit_exact():
    """The constructed mesh of exact ties: every half-ray of the GPU tracer equals the
    oracle's (smaller distance, then smaller projection, then smaller index)."""
    from test_oracle_pins import _tie_mesh
    m = _tie_mesh()
    o = Oracle(m)
    ctx = gpu_context(m, oracle_dirs=o.dirs)
    ctx.trace_rays()
    for p in range(m.n):
        for r in range(o.dirs.shape[0]):
            t = o.trace(p, r)
            g = ctx.get_ray(p, r)
            assert g["cells"].tolist() == t["cells"].tolist(), (p, r)
            assert np.array_equal(g["ds"], t["ds"]), (p, r)


@pytest.mark.parametrize("precision", [0, 1])
def test_opacity_floor_slab_matches_oracle(precision):
    """The slab of the oracle's floor pin (a line negligible against chi_min = 1e-12 and
    3e-12 m^-1, no boundary radiation): the GPU's J, L and J_eff equal the oracle's
    (1e-10 FP64, 1e-4 mixed), so both carry the line's emission through the floor."""
    sp = syn.species_two_level()
    a = 2e11
    m = syn.model_line_1d(np.linspace(-a, a, 161), 0.0, 1e10, 30.0, 150.0, 1e-16, sp, 7)
    for chi in (1e-12, 3e-12):
        o = Oracle(m, chi_min=chi, T_cmb=0.01)
        ctx = gpu_context(m, oracle_dirs=o.dirs, precision=precision, chi_min=chi, T_cmb=0.01)
        ctx.trace_rays()
        ctx.init_populations()
        ctx.formal_solve()
        J, L, E = ctx.get_radiation()
        Jo, Lo, Eo = o.formal_solve(o.lte())
        tol = TOL64 if precision == 0 else 1e-4
        assert np.max(rel_err(J, Jo)) < tol
        assert np.max(rel_err(E, Eo)) < tol
        assert np.max(np.abs(L - Lo)) < tol * float(np.max(np.abs(Lo)))
