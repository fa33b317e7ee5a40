"""Seeded synthetic models shaped like the paper's test and application models.

All quantities are SI: metres, m/s, kelvin, m^-3, joules, s^-1, m^3 s^-1.
Random numbers come from numpy's PCG64 (``np.random.default_rng(seed)``).

Shapes follow the paper's workloads:
  * spherically symmetric clouds with n ~ r^-2 (van Zadelhoff problem 1, Sec. 4.2.1);
  * 3D clumpy clouds with a radial outflow (velocity law of Sec. 4.2.2);
  * a flared Keplerian disc (Sec. 5);
  * the semi-analytic 1D line models (Sec. 4.1: Hubble-Lemaitre and power-law).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# CODATA 2018 exact / recommended values, used by the generators only to convert
# wavenumbers and temperatures into SI inputs.
CODATA = dict(h=6.62607015e-34, kB=1.380649e-23, c=299792458.0, amu=1.66053906660e-27)
AU = 1.495978707e11
G_GRAV = 6.67430e-11
M_SUN = 1.98847e30

GEOM_3D = 0
GEOM_SPHERICAL_1D = 1


@dataclasses.dataclass
class Species:
    """Level/line/collision tables of one species (synthetic stand-in for LAMDA data)."""
    E: np.ndarray          # [n_lev] level energies, J
    g: np.ndarray          # [n_lev] statistical weights
    mass: float            # kg
    up: np.ndarray         # [n_lines] int32 upper level of each radiative line
    lo: np.ndarray         # [n_lines] int32 lower level
    A: np.ndarray          # [n_lines] Einstein A, s^-1
    T_grid: np.ndarray     # [n_T] K
    K_down: np.ndarray     # [n_lev*(n_lev-1)/2][n_T] de-excitation coefficients, m^3 s^-1,
                           # pair order (i>j): (1,0),(2,0),(2,1),(3,0),...

    @property
    def n_lev(self):
        return int(self.E.shape[0])

    @property
    def n_lines(self):
        return int(self.A.shape[0])


@dataclasses.dataclass
class Model:
    """A point cloud with neighbour lists and per-point physical fields."""
    name: str
    pos: np.ndarray        # [n][3] m
    vel: np.ndarray        # [n][3] m/s
    nbr_off: np.ndarray    # [n+1] int64 CSR offsets
    nbr_idx: np.ndarray    # [E] int32 neighbour indices
    is_bdy: np.ndarray     # [n] uint8
    n_coll: np.ndarray     # [n] collision-partner (H2) density, m^-3
    T: np.ndarray          # [n] K
    v_turb: np.ndarray     # [n] m/s
    n_spec: np.ndarray     # [n] species density, m^-3
    species: Species
    geometry: int = GEOM_3D
    nside: int = 1                     # HEALPix resolution for the ray directions
    n_q: int = 31                      # Gauss-Hermite points per line
    dirs: np.ndarray | None = None     # custom directions [R][3] (overrides nside)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self):
        return int(self.pos.shape[0])


# --------------------------------------------------------------------------- species
def species_two_level(A21=1.0e-4, K21=2.0e-16, dE_cm=6.0, g_ratio=3.0, mass_amu=1.0):
    """The fictitious 2-level species of the paper's semi-analytic tests and of
    van Zadelhoff problem 1 (Table 'test_species'): E2-E1 = 6.0 cm^-1, g2/g1 = 3,
    A21 = 1e-4 s^-1, K21 = 2e-10 cm^3 s^-1 = 2e-16 m^3 s^-1. Its mass is 1 amu (the
    mass for which the printed line widths 519.03 kHz and 357.53 kHz follow)."""
    h, c = CODATA["h"], CODATA["c"]
    E = np.array([0.0, h * c * dE_cm * 100.0])
    g = np.array([1.0, g_ratio])
    T_grid = np.array([5.0, 1000.0])
    K_down = np.full((1, 2), K21)
    return Species(E=E, g=g, mass=mass_amu * CODATA["amu"], up=np.array([1], np.int32),
                   lo=np.array([0], np.int32), A=np.array([A21]), T_grid=T_grid, K_down=K_down)


def species_ladder(n_lev, dE_cm=6.0, A1=1.0e-5, K0=1.0e-16, mass_amu=28.0):
    """Equally spaced levels E_i = i dE, g_i = 2i + 1, radiative lines i -> i-1 only, all
    at the same frequency: every line overlaps every other one, so a frequency bin sums
    all their profiles. A_i = A1 i; collisional de-excitation K0 / 10^(i-j-1), constant
    in T."""
    h, c = CODATA["h"], CODATA["c"]
    E = np.arange(n_lev) * h * c * dE_cm * 100.0
    g = 2.0 * np.arange(n_lev) + 1.0
    up = np.arange(1, n_lev, dtype=np.int32)
    lo = up - 1
    A = A1 * up.astype(np.float64)
    T_grid = np.array([5.0, 1000.0])
    K = [K0 / 10.0 ** (i - j - 1) for i in range(1, n_lev) for j in range(i)]
    K_down = np.repeat(np.array(K)[:, None], 2, axis=1)
    return Species(E=E, g=g, mass=mass_amu * CODATA["amu"], up=up, lo=lo, A=A, T_grid=T_grid, K_down=K_down)


def species_rotor(n_lev, rng, mass_amu=28.0, B_range=(40e9, 60e9), A1_scale=1e-7,
                  a_range=(1e-17, 1e-16), b_range=(0.0, 0.5), dj_decay=10.0):
    """Seeded linear-rotor ladder: E_J = h B J(J+1), g_J = 2J+1, radiative lines
    J -> J-1 with A_J = A_1 J^3, and de-excitation coefficients for every pair J > J'
    K(T) = a (T / 100 K)^b / dj_decay^(J - J' - 1) tabulated on a temperature grid.
    Collisions are dominated by Delta J = 1: with strong Delta J >= 2 excitation the fast
    radiative cascade (A ~ J^3) inverts the lowest line at low density (a maser)."""
    h = CODATA["h"]
    B = rng.uniform(*B_range)
    J = np.arange(n_lev, dtype=np.float64)
    E = h * B * J * (J + 1.0)
    g = 2.0 * J + 1.0
    A1 = A1_scale * np.exp(rng.uniform(np.log(0.5), np.log(2.0)))
    up = np.arange(1, n_lev, dtype=np.int32)
    lo = up - 1
    A = A1 * up.astype(np.float64) ** 3
    a = np.exp(rng.uniform(np.log(a_range[0]), np.log(a_range[1])))
    b = rng.uniform(*b_range)
    T_grid = np.array([5.0, 10.0, 20.0, 50.0, 100.0, 200.0, 500.0, 1000.0, 3000.0])
    rows = []
    for i in range(1, n_lev):
        for j in range(i):
            rows.append(a * (T_grid / 100.0) ** b / dj_decay ** (i - j - 1))
    return Species(E=E, g=g, mass=mass_amu * CODATA["amu"], up=up, lo=lo, A=A,
                   T_grid=T_grid, K_down=np.array(rows))


# --------------------------------------------------------------------------- meshes
def knn_symmetric(pos, k):
    """k-nearest-neighbour lists made symmetric (i in N(j) <=> j in N(i)), as CSR with
    each row sorted by index."""
    from scipy.spatial import cKDTree
    n = pos.shape[0]
    kk = min(k + 1, n)
    _, idx = cKDTree(pos).query(pos, k=kk)
    idx = np.asarray(idx).reshape(n, kk)
    rows = np.repeat(np.arange(n), kk - 1)
    cols = idx[:, 1:].reshape(-1)
    keep = cols != rows
    rows, cols = rows[keep], cols[keep]
    a = np.concatenate([rows, cols])
    b = np.concatenate([cols, rows])
    key = np.unique(a.astype(np.int64) * n + b)
    a = key // n
    b = key % n
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, a + 1, 1)
    off = np.cumsum(off)
    return off, b.astype(np.int32)


def _morton_order(pos):
    """Permutation that sorts points along a 3D Morton (Z-order) curve."""
    lo = pos.min(0)
    span = np.maximum(pos.max(0) - lo, 1e-300)
    q = np.clip(((pos - lo) / span * 1023.0).astype(np.int64), 0, 1023)
    code = np.zeros(pos.shape[0], np.int64)
    for bit in range(10):
        for ax in range(3):
            code |= ((q[:, ax] >> bit) & 1) << (3 * bit + ax)
    return np.argsort(code, kind="stable")


def _fibonacci_sphere(m, radius):
    i = np.arange(m) + 0.5
    z = 1.0 - 2.0 * i / m
    phi = np.pi * (1.0 + 5.0 ** 0.5) * i
    s = np.sqrt(1.0 - z * z)
    return radius * np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)


def _finish(name, pos, vel, is_bdy, fields, species, k, nside, n_q, meta, sort=True):
    if sort:
        perm = _morton_order(pos)
        pos, vel, is_bdy = pos[perm], vel[perm], is_bdy[perm]
        fields = {key: v[perm] for key, v in fields.items()}
    off, idx = knn_symmetric(pos, k)
    return Model(name=name, pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel),
                 nbr_off=off, nbr_idx=idx, is_bdy=is_bdy.astype(np.uint8),
                 n_coll=fields["n_coll"], T=fields["T"], v_turb=fields["v_turb"],
                 n_spec=fields["n_spec"], species=species, geometry=GEOM_3D,
                 nside=nside, n_q=n_q, meta=meta)


def model_sphere_1d(seed=0, n=200, r_min=1e12, r_max=1e15, n_q=31, nside=1, A21=None,
                    abundance=1e-8):
    """Spherically symmetric cloud: n points on a log radial grid, n_H2 = n0 (r/r_min)^-2
    with n0 log-uniform in [1e9, 1e12] m^-3, T = 20 K, X = 1e-8, no bulk velocity,
    150 m/s turbulence, 2-level species with A21 log-uniform around 1e-5 s^-1 and a
    constant collisional coefficient. Geometry: one point per radius on the +z axis."""
    rng = np.random.default_rng(seed)
    r = np.geomspace(r_min, r_max, n)
    n0 = np.exp(rng.uniform(np.log(1e9), np.log(1e12)))
    if A21 is None:
        A21 = 1e-5 * np.exp(rng.uniform(np.log(0.5), np.log(2.0)))
    sp = species_two_level(A21=A21)
    pos = np.zeros((n, 3))
    pos[:, 2] = r
    vel = np.zeros((n, 3))
    n_h2 = n0 * (r / r_min) ** -2
    off = np.zeros(n + 1, np.int64)
    nb = []
    for i in range(n):
        row = [j for j in (i - 1, i + 1) if 0 <= j < n]
        nb.extend(row)
        off[i + 1] = off[i] + len(row)
    is_bdy = np.zeros(n, np.uint8)
    is_bdy[-1] = 1
    return Model(name="sphere1d", pos=pos, vel=vel, nbr_off=off,
                 nbr_idx=np.array(nb, np.int32), is_bdy=is_bdy, n_coll=n_h2,
                 T=np.full(n, 20.0), v_turb=np.full(n, 150.0), n_spec=abundance * n_h2,
                 species=sp, geometry=GEOM_SPHERICAL_1D, nside=nside, n_q=n_q,
                 meta=dict(seed=seed, n0=n0, A21=A21))


def model_clumpy_3d(seed=0, n=50_000, R=1e15, n_clumps=20, k=16, nside=2, n_q=31,
                    n_lev=5, v_max=1.0e4, bdy_frac=None, n_h2_ref=1e11, abundance=1e-6,
                    species=None):
    """3D clumpy cloud: points drawn from an r^-2 background plus seeded Gaussian clumps
    inside a sphere of radius R, about bdy_frac of them on the bounding sphere (convex
    hull), symmetric k-NN lists, T falling log-linearly from 100 K (centre) to 10 K
    (edge), radial outflow v = v_max r/R, 150 m/s turbulence, seeded linear rotor.
    By default the boundary points get the spacing of the interior points at the edge.
    The default density (n_H2 = 1e11 m^-3 (r/R)^-2 plus clumps) and abundance (1e-6) make
    the lines optically thick without population inversion of the rotor's lowest line,
    which sets in below ~1e10 m^-3 (a maser the method does not treat)."""
    rng = np.random.default_rng(seed)
    if bdy_frac is None:
        nb_est = 0.7 * n
        for _ in range(3):
            spacing = (4.0 * np.pi * 0.97 / (0.7 * (n - nb_est))) ** (1.0 / 3.0)
            nb_est = 4.0 * np.pi / spacing ** 2
        n_b = max(12, int(round(nb_est)))
    else:
        n_b = max(12, int(round(bdy_frac * n)))
    n_i = n - n_b
    cdir = rng.normal(size=(n_clumps, 3))
    cdir /= np.linalg.norm(cdir, axis=1, keepdims=True)
    cc = cdir * rng.uniform(0.0, 0.7, (n_clumps, 1)) * R
    cs = rng.uniform(0.02, 0.10, n_clumps) * R
    ca = np.exp(rng.uniform(np.log(1.0), np.log(100.0), n_clumps))
    n_clump_pts = int(0.3 * n_i)
    n_bg = n_i - n_clump_pts
    # r^-2 point density in 3D <=> radius uniform in r
    rr = rng.uniform(0.01 * R, 0.98 * R, n_bg)
    d = rng.normal(size=(n_bg, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    bg = rr[:, None] * d
    w = ca * cs ** 3
    which = rng.choice(n_clumps, size=n_clump_pts, p=w / w.sum())
    cl = cc[which] + rng.normal(size=(n_clump_pts, 3)) * cs[which, None]
    rc = np.linalg.norm(cl, axis=1)
    bad = rc > 0.98 * R
    for _ in range(50):
        if not bad.any():
            break
        cl[bad] = cc[which[bad]] + rng.normal(size=(bad.sum(), 3)) * cs[which[bad], None]
        rc = np.linalg.norm(cl, axis=1)
        bad = rc > 0.98 * R
    if bad.any():   # leftovers come from the background distribution
        nb = int(bad.sum())
        db = rng.normal(size=(nb, 3))
        db /= np.linalg.norm(db, axis=1, keepdims=True)
        cl[bad] = rng.uniform(0.01 * R, 0.98 * R, (nb, 1)) * db
    pos = np.concatenate([bg, cl, _fibonacci_sphere(n_b, R)])
    is_bdy = np.zeros(n, np.uint8)
    is_bdy[n_i:] = 1
    r = np.linalg.norm(pos, axis=1)
    rhat = pos / np.maximum(r, 1e-300)[:, None]
    dens = (np.maximum(r, 0.01 * R) / R) ** -2
    for c0, s0, a0 in zip(cc, cs, ca):
        dens = dens + a0 * np.exp(-0.5 * np.sum((pos - c0) ** 2, 1) / s0 ** 2)
    n_h2 = n_h2_ref * dens
    T = 100.0 * (10.0 / 100.0) ** (r / R)
    vel = v_max * (r / R)[:, None] * rhat
    sp = species if species is not None else species_rotor(n_lev, rng)
    fields = dict(n_coll=n_h2, T=T, v_turb=np.full(n, 150.0), n_spec=abundance * n_h2)
    return _finish("clumpy3d", pos, vel, is_bdy, fields, sp, k, nside, n_q,
                   dict(seed=seed, R=R))


def model_disc(seed=0, n=200_000, r_in_au=10.0, r_out_au=200.0, k=16, nside=4, n_q=63,
               n_lev=20, bdy_frac=0.02, env_frac=0.1, n_h2_in=1e13, abundance=1e-4, T_in=100.0):
    """Flared Keplerian disc: n ~ r^-1 exp(-z^2/2H^2) with H = 0.1 r, T ~ r^-0.5,
    v = sqrt(G M_sun / r) phi_hat, boundary points on the bounding sphere, 20-level rotor."""
    rng = np.random.default_rng(seed)
    r_in, r_out = r_in_au * AU, r_out_au * AU
    n_b = max(12, int(round(bdy_frac * n)))
    n_env = int(round(env_frac * n))
    n_i = n - n_b - n_env
    # surface density ~ r^-1 * H ~ r^0 -> radius uniform in area weighting r dr: p(r) ~ r
    rr = np.sqrt(rng.uniform(r_in ** 2, (0.97 * r_out) ** 2, n_i))
    ph = rng.uniform(0, 2 * np.pi, n_i)
    z = rng.normal(size=n_i) * 0.1 * rr
    z = np.clip(z, -0.4 * rr, 0.4 * rr)
    pos_i = np.stack([rr * np.cos(ph), rr * np.sin(ph), z], 1)
    # a sparse envelope filling the bounding sphere (the floor density), so that rays
    # leaving the disc reach the boundary instead of ending at a dead end
    d = rng.normal(size=(n_env, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos_e = d * (0.97 * r_out * rng.uniform(0, 1, (n_env, 1)) ** (1.0 / 3.0))
    pos = np.concatenate([pos_i, pos_e, _fibonacci_sphere(n_b, r_out)])
    is_bdy = np.zeros(n, np.uint8)
    is_bdy[n_i + n_env:] = 1
    rc = np.maximum(np.hypot(pos[:, 0], pos[:, 1]), r_in)
    H = 0.1 * rc
    n_h2 = n_h2_in * (rc / r_in) ** -1 * np.exp(-0.5 * (pos[:, 2] / H) ** 2)
    n_h2 = np.maximum(n_h2, 1e-6 * n_h2_in)
    T = T_in * (rc / r_in) ** -0.5
    vk = np.sqrt(G_GRAV * M_SUN / rc)
    phat = np.stack([-pos[:, 1], pos[:, 0], np.zeros(n)], 1) / rc[:, None]
    vel = vk[:, None] * phat
    sp = species_rotor(n_lev, rng)
    fields = dict(n_coll=n_h2, T=T, v_turb=np.full(n, 150.0), n_spec=abundance * n_h2)
    return _finish("disc", pos, vel, is_bdy, fields, sp, k, nside, n_q, dict(seed=seed))


def model_batch(seed=0, n_models=64, n_range=(2000, 40000), **kw):
    """Independent clumpy clouds of uneven size (log-uniform point counts)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]), n_models))
    sizes = sizes.astype(int)
    return [model_clumpy_3d(seed=seed * 1000 + i, n=int(s), v_max=rng.uniform(2e3, 2e4), **kw)
            for i, s in enumerate(sizes)]


def model_line_1d(x, vel_z, n_h2, T, v_turb, abundance, species, n_q):
    """Points on the z axis (a single line) with neighbours i-1, i+1, both ends on the
    boundary, and the two ray directions +z and -z (the paper's 1D semi-analytic setup:
    one ray pair through the whole model)."""
    n = x.shape[0]
    pos = np.zeros((n, 3))
    pos[:, 2] = x
    vel = np.zeros((n, 3))
    vel[:, 2] = vel_z
    off = np.zeros(n + 1, np.int64)
    nb = []
    for i in range(n):
        row = [j for j in (i - 1, i + 1) if 0 <= j < n]
        nb.extend(row)
        off[i + 1] = off[i] + len(row)
    is_bdy = np.zeros(n, np.uint8)
    is_bdy[0] = is_bdy[-1] = 1
    f = lambda v: np.broadcast_to(np.asarray(v, np.float64), (n,)).copy()
    return Model(name="line1d", pos=pos, vel=vel, nbr_off=off, nbr_idx=np.array(nb, np.int32),
                 is_bdy=is_bdy, n_coll=f(n_h2), T=f(T), v_turb=f(v_turb),
                 n_spec=f(n_h2) * abundance, species=species, geometry=GEOM_3D, n_q=n_q,
                 dirs=np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]))


def hubble_line_1d(n_cells=100, R=495e3, c_dbeta=0.01, n_q=100):
    """Homogeneous Hubble-Lemaitre test on a uniform grid in [-R, R] (Sec. 4.1.1):
    v = c dbeta z, n_H2 = 1e12 m^-3, X = 1e-4, T = 45 K, no turbulence."""
    x = np.linspace(-R, R, n_cells)
    return model_line_1d(x, c_dbeta * x, 1e12, 45.0, 0.0, 1e-4, species_two_level(), n_q)


def hubble_sphere_1d(n_shells=50, R=495e3, c_dbeta=0.01, n_q=100, nside=1):
    """Homogeneous Hubble-Lemaitre sphere as spherically symmetric shells, radii
    uniform in [0, R] (the first shell is the centre point)."""
    r = np.linspace(0.0, R, n_shells)
    n = n_shells
    pos = np.zeros((n, 3)); pos[:, 2] = r
    vel = np.zeros((n, 3)); vel[:, 2] = c_dbeta * r
    off = np.zeros(n + 1, np.int64); nb = []
    for i in range(n):
        row = [j for j in (i - 1, i + 1) if 0 <= j < n]
        nb.extend(row); off[i + 1] = off[i] + len(row)
    is_bdy = np.zeros(n, np.uint8); is_bdy[-1] = 1
    return Model(name="hubble_sphere", pos=pos, vel=vel, nbr_off=off,
                 nbr_idx=np.array(nb, np.int32), is_bdy=is_bdy, n_coll=np.full(n, 1e12),
                 T=np.full(n, 45.0), v_turb=np.zeros(n), n_spec=np.full(n, 1e8),
                 species=species_two_level(), geometry=GEOM_SPHERICAL_1D, nside=nside, n_q=n_q)


def powerlaw_line_1d(n_shells=50, R_in=1e13, R=7.8e16, n_in=2e13, abundance=1e-6, n_q=100):
    """Power-law density with an empty core (Sec. 4.1.2) as a single line through the
    centre: shells log-spaced in [R_in, R] on both sides, n = n_in (R_in/r)^2, T = 20 K,
    150 m/s turbulence, no velocity field."""
    r = np.geomspace(R_in, R, n_shells)
    x = np.concatenate([-r[::-1], r])
    n_h2 = n_in * (R_in / np.abs(x)) ** 2
    return model_line_1d(x, np.zeros_like(x), n_h2, 20.0, 150.0, abundance,
                         species_two_level(), n_q)


def model_tiny_3d(seed=0, n=20, k=6, nside=1, n_q=7, n_lev=3, v_max=3e3):
    """A handful of random points in a unit-ish ball, with 8+ boundary points on the
    bounding sphere; used for brute-force checks."""
    rng = np.random.default_rng(seed)
    R = 1e13
    n_b = max(8, n // 3)
    n_i = n - n_b
    d = rng.normal(size=(n_i, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.concatenate([d * rng.uniform(0.05, 0.9, (n_i, 1)) * R, _fibonacci_sphere(n_b, R)])
    is_bdy = np.zeros(n, np.uint8); is_bdy[n_i:] = 1
    r = np.linalg.norm(pos, axis=1)
    vel = v_max * pos / R
    n_h2 = 1e10 * np.exp(rng.uniform(-1, 1, n))
    sp = species_rotor(n_lev, rng)
    fields = dict(n_coll=n_h2, T=rng.uniform(15, 60, n), v_turb=np.full(n, 150.0),
                  n_spec=1e-6 * n_h2)
    return _finish("tiny3d", pos, vel, is_bdy, fields, sp, k, nside, n_q, dict(seed=seed), sort=False)


def model_lattice_3d(m=7, spacing=1e12, n_q=7):
    """Cubic lattice m^3 with 26-neighbour lists; the outer layer is the boundary.
    Rays along the axes must follow lattice lines exactly."""
    ax = (np.arange(m) - (m - 1) / 2.0) * spacing
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n = pos.shape[0]
    ijk = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    off = np.zeros(n + 1, np.int64); nb = []
    for p in range(n):
        i, j, kk = ijk[p]
        row = []
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    if di == dj == dk == 0:
                        continue
                    a, b, c = i + di, j + dj, kk + dk
                    if 0 <= a < m and 0 <= b < m and 0 <= c < m:
                        row.append((a * m + b) * m + c)
        nb.extend(sorted(row)); off[p + 1] = off[p] + len(row)
    is_bdy = ((ijk == 0) | (ijk == m - 1)).any(1).astype(np.uint8)
    sp = species_two_level()
    return Model(name="lattice", pos=pos, vel=np.zeros((n, 3)), nbr_off=off,
                 nbr_idx=np.array(nb, np.int32), is_bdy=is_bdy, n_coll=np.full(n, 1e10),
                 T=np.full(n, 20.0), v_turb=np.full(n, 150.0), n_spec=np.full(n, 1.0),
                 species=sp, geometry=GEOM_3D, n_q=n_q,
                 dirs=np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 1.0, 0], [0, -1.0, 0],
                                [0, 0, 1.0], [0, 0, -1.0]]))


def shell_counts(radii, n_cells, floor=12):
    """Points per shell for a shell mesh of n_cells points: proportional to r^2 (a
    uniform point density), at least `floor` per shell, the rounding remainder taken
    up by the outermost shell."""
    r2 = np.asarray(radii, np.float64) ** 2
    lo, hi = 0.0, float(n_cells) / r2.max() * 2.0
    for _ in range(200):   # bisect the scale so that the counts sum to about n_cells
        mid = 0.5 * (lo + hi)
        s = np.maximum(floor, np.round(mid * r2)).sum()
        lo, hi = (mid, hi) if s < n_cells else (lo, mid)
    cnt = np.maximum(floor, np.round(lo * r2)).astype(np.int64)
    cnt[-1] += n_cells - cnt.sum()
    return cnt


def shells_3d(radii, n_cells, seed=0, k=16):
    """A 3D point mesh made of spherical shells (the paper's mapping of a 1D radial
    grid to 3D, Sec. 4.1): shell i is a Fibonacci lattice of shell_counts() points at
    radius radii[i], each turned by a seeded random rotation; the outermost shell is the
    boundary. Returns positions, boundary flags and the shell index of every point."""
    rng = np.random.default_rng(seed)
    cnt = shell_counts(radii, n_cells)
    pos, shell = [], []
    for i, (r, m) in enumerate(zip(radii, cnt)):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        pos.append(_fibonacci_sphere(int(m), r) @ q.T)
        shell.append(np.full(int(m), i))
    pos = np.concatenate(pos)
    shell = np.concatenate(shell)
    is_bdy = (shell == len(radii) - 1).astype(np.uint8)
    return pos, is_bdy, shell


def hubble_shells_3d(n_shells=50, n_cells=12_528, R=495e3, c_dbeta=0.01, n_q=100, nside=4,
                     k=16, seed=0):
    """3D Hubble-Lemaitre model of the paper's test table (Sec. 4.1.1): the radii of the
    uniform 1D grid of 2 n_shells cells in [-R, R] as shells of 3D points (n_cells in
    all), v = c dbeta x, n_H2 = 1e12 m^-3, X = 1e-4, T = 45 K, no turbulence, the 2-level
    species of the paper's Table 'test_species'."""
    x = np.linspace(-R, R, 2 * n_shells)
    radii = x[n_shells:]
    pos, is_bdy, shell = shells_3d(radii, n_cells, seed=seed)
    n = pos.shape[0]
    fields = dict(n_coll=np.full(n, 1e12), T=np.full(n, 45.0), v_turb=np.zeros(n),
                  n_spec=np.full(n, 1e8))
    m = _finish("hubble_shells", pos, c_dbeta * pos, is_bdy, fields, species_two_level(), k,
                nside, n_q, dict(seed=seed, R=R, c_dbeta=c_dbeta))
    return m


def vz_problem1(abundance=1e-6, v_inf=0.0, gamma=0.5, n_shells=50, R_in=1e13, R=7.8e16,
                n_in=2e13, n_q=31, nside=2):
    """Van Zadelhoff et al. (2002) problem 1 as used in the paper (Sec. 4.2.1, 4.2.2): the
    power-law cloud n_H2 = n_in (R_in/r)^2 on n_shells log-spaced radii in [R_in, R]
    with an empty core, T = 20 K, 150 m/s turbulence, the 2-level species of Table
    'test_species', X = 1e-8 (problem 1a) or 1e-6 (1b), and the radial outflow
    v = v_inf ((r - R_in)/(R - R_in))^gamma of problems 1c/1d (v_inf = 0: 1a/1b).
    Spherically symmetric geometry (one point per radius on the +z axis)."""
    r = np.geomspace(R_in, R, n_shells)
    m = model_sphere_1d(n=n_shells, r_min=R_in, r_max=R, n_q=n_q, nside=nside, A21=1.0e-4,
                        abundance=abundance)
    m.n_coll = n_in * (R_in / r) ** 2
    m.n_spec = abundance * m.n_coll
    m.T = np.full(n_shells, 20.0)
    m.v_turb = np.full(n_shells, 150.0)
    m.vel = np.zeros((n_shells, 3))
    m.vel[:, 2] = v_inf * ((r - R_in) / (R - R_in)) ** gamma
    m.name = "vz_p1"
    m.meta = dict(abundance=abundance, v_inf=v_inf, gamma=gamma)
    return m
