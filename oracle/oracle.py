"""Python side of the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Holds the parts of the method that are plain closed formulas, written with numpy:
  * HEALPix ring-scheme pixel centres (Gorski et al. 2005), the paper's ray directions
    (Sec. 3.1.3);
  * Gauss-Hermite roots and the paper's weight formula (Sec. 3.1.2);
and a ctypes binding to ``magritte_oracle.c`` (ray tracing, Feautrier solve,
statistical equilibrium, ALI, Ng). The CUDA path shares none of this code.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")

CONST = dict(h=6.62607015e-34, kB=1.380649e-23, c=299792458.0, amu=1.66053906660e-27,
             T_cmb=2.725)


def lib_path():
    return os.path.join(BUILD, "liboracle.so")


def build_oracle(force=False):
    """Compile the C oracle (gcc, no FMA contraction, OpenMP)."""
    os.makedirs(BUILD, exist_ok=True)
    out = lib_path()
    src = os.path.join(HERE, "magritte_oracle.c")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


# ------------------------------------------------------------------ closed formulas
def planck(nu, T):
    """Black-body intensity B_nu(T)."""
    h, k, c = CONST["h"], CONST["kB"], CONST["c"]
    return 2.0 * h * nu ** 3 / c ** 2 / np.expm1(h * nu / (k * T))


def line_width_nu(nu, T, mass, v_turb):
    """delta_nu = nu/c sqrt(2kT/m + v_turb^2) (Sec. 2.2.1)."""
    return nu / CONST["c"] * np.sqrt(2.0 * CONST["kB"] * T / mass + v_turb ** 2)


def healpix_dirs(nside):
    """Unit vectors of the 12 nside^2 HEALPix pixel centres in RING order, from the
    pixel-to-angle formulas of Gorski et al. (2005) (polar caps and equatorial belt)."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    z = np.empty(npix)
    phi = np.empty(npix)
    for p in range(npix):
        if p < ncap:                       # north polar cap
            i = int((1 + math.isqrt(1 + 2 * p)) // 2)
            while 2 * i * (i - 1) > p:
                i -= 1
            while 2 * (i + 1) * i <= p:
                i += 1
            j = p + 1 - 2 * i * (i - 1)
            z[p] = 1.0 - i * i / (3.0 * nside * nside)
            phi[p] = math.pi / (2.0 * i) * (j - 0.5)
        elif p < npix - ncap:              # equatorial belt
            pp = p - ncap
            i = pp // (4 * nside) + nside
            j = pp % (4 * nside) + 1
            s = (i - nside + 1) % 2
            z[p] = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            phi[p] = math.pi / (2.0 * nside) * (j - s / 2.0)
        else:                              # south polar cap
            pp = npix - p
            i = int((1 + math.isqrt(2 * pp - 1)) // 2)
            while 2 * i * (i - 1) >= pp:
                i -= 1
            while 2 * (i + 1) * i < pp:
                i += 1
            j = 4 * i + 1 - (pp - 2 * i * (i - 1))
            z[p] = -1.0 + i * i / (3.0 * nside * nside)
            phi[p] = math.pi / (2.0 * i) * (j - 0.5)
    st = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], 1)


def antipodes(dirs, tol=1e-12):
    """Index of the direction opposite to each direction (exhaustive search)."""
    R = dirs.shape[0]
    out = np.full(R, -1, np.int32)
    for r in range(R):
        d = np.linalg.norm(dirs + dirs[r], axis=1)
        k = int(np.argmin(d))
        if d[k] > tol:
            raise ValueError(f"direction {r} has no antipode")
        out[r] = k
    return out


def _hermite_phys(n, x):
    """Physicists' Hermite polynomial H_n(x) from H_{k+1} = 2x H_k - 2k H_{k-1}."""
    h0, h1 = np.ones_like(x), 2.0 * x
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, 2.0 * x * h1 - 2.0 * k * h0
    return h1


def gauss_hermite(Q):
    """Roots r_n of H_Q and the paper's weights w_n = 2^(Q-1) Q! / (Q H_{Q-1}(r_n))^2
    (Sec. 3.1.2), which sum to one (profile-normalised). Roots come from numpy's
    Gauss-Hermite routine and are refined by Newton steps on H_Q; the weights are
    evaluated in log form to stay in range for large Q."""
    from numpy.polynomial.hermite import hermgauss
    r, _ = hermgauss(Q)
    for _ in range(3):
        Hq = _hermite_phys(Q, r)
        dHq = 2.0 * Q * _hermite_phys(Q - 1, r)
        r = r - Hq / dHq
    Hm = _hermite_phys(Q - 1, r)
    logw = (Q - 1) * math.log(2.0) + math.lgamma(Q + 1) - 2.0 * (math.log(Q) + np.log(np.abs(Hm)))
    return r, np.exp(logw)


# ------------------------------------------------------------------ ctypes binding
class OrModel(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("geometry", C.c_int32), ("pad0", C.c_int32),
        ("pos", C.c_void_p), ("vel", C.c_void_p), ("nbr_off", C.c_void_p), ("nbr_idx", C.c_void_p),
        ("is_bdy", C.c_void_p), ("n_coll", C.c_void_p), ("T", C.c_void_p), ("v_turb", C.c_void_p),
        ("n_spec", C.c_void_p),
        ("n_lev", C.c_int32), ("n_lines", C.c_int32), ("E", C.c_void_p), ("g", C.c_void_p),
        ("mass", C.c_double), ("up", C.c_void_p), ("lo", C.c_void_p), ("A", C.c_void_p),
        ("n_T", C.c_int32), ("pad1", C.c_int32), ("T_grid", C.c_void_p), ("K_down", C.c_void_p),
        ("R", C.c_int32), ("Q", C.c_int32), ("dirs", C.c_void_p), ("antipode", C.c_void_p),
        ("roots", C.c_void_p), ("weights", C.c_void_p),
        ("dshift_frac", C.c_double), ("chi_min", C.c_double), ("dtau_min", C.c_double),
        ("T_cmb", C.c_double), ("max_steps", C.c_int64),
    ]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(build_oracle())
        P = C.c_void_p
        L.or_trace.argtypes = [P, C.c_int64, C.c_int, C.c_int64, P, P, P, P, P, P]
        L.or_lte.argtypes = [P, P]
        L.or_formal_solve.argtypes = [P, P, C.c_int64, P, P, P, P, P, C.c_int]
        L.or_stateq.argtypes = [P, P, P, P, P, P]
        L.or_max_rel_change.argtypes = [P, P, P]
        L.or_max_rel_change.restype = C.c_double
        L.or_ng.argtypes = [C.c_int64, P, P, P, P, P]
        L.or_ali.argtypes = [P, P, C.c_double, C.c_int, C.c_int, P, P, C.c_int]
        L.or_feautrier.argtypes = [C.c_int64, C.c_int64, P, P, C.c_double, C.c_double, P, P, P]
        L.or_trace_all.argtypes = [P, C.c_int64, P, P, P, P, P, P, P, P, C.c_int]
        L.or_width.argtypes = [P, C.c_int64]
        L.or_width.restype = C.c_double
        L.or_image.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P, C.c_int64, P, P, P, C.c_int]
        L.or_first_order.argtypes = [C.c_int64, P, P, C.c_double]
        L.or_first_order.restype = C.c_double
        L.or_feautrier_band.argtypes = [C.c_int64, C.c_int64, C.c_int64, P, P, P]
        L.or_formal_solve_band.argtypes = [P, P, C.c_int64, P, C.c_int, P, P, P, P, P, C.c_int]
        L.or_band_geometry.argtypes = [P, C.c_int64, P, C.c_int, P, P, P]
        L.or_cell_generator.argtypes = [P, C.c_int64, P, P, P]
        L.or_formal_solve_sca.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, C.c_int]
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """FP64 oracle bound to one synthetic model (``synthetic.Model``)."""

    def __init__(self, model, dirs=None, Q=None, dshift_frac=1.0 / 3.0, chi_min=1e-30,
                 dtau_min=1e-30, T_cmb=2.725, max_steps=100000, nthreads=0):
        self.model = model
        sp = model.species
        if dirs is None:
            dirs = model.dirs if model.dirs is not None else healpix_dirs(model.nside)
        self.dirs = np.ascontiguousarray(dirs, np.float64)
        self.anti = antipodes(self.dirs)
        self.Q = int(Q if Q is not None else model.n_q)
        self.roots, self.weights = gauss_hermite(self.Q)
        self.nthreads = nthreads
        f = lambda a, t=np.float64: np.ascontiguousarray(a, t)
        self._keep = dict(
            pos=f(model.pos), vel=f(model.vel), nbr_off=f(model.nbr_off, np.int64),
            nbr_idx=f(model.nbr_idx, np.int32), is_bdy=f(model.is_bdy, np.uint8),
            n_coll=f(model.n_coll), T=f(model.T), v_turb=f(model.v_turb), n_spec=f(model.n_spec),
            E=f(sp.E), g=f(sp.g), up=f(sp.up, np.int32), lo=f(sp.lo, np.int32), A=f(sp.A),
            T_grid=f(sp.T_grid), K_down=f(sp.K_down), dirs=self.dirs, anti=self.anti,
            roots=f(self.roots), weights=f(self.weights))
        k = self._keep
        self.m = OrModel(
            n=model.n, geometry=model.geometry, pos=_ptr(k["pos"]), vel=_ptr(k["vel"]),
            nbr_off=_ptr(k["nbr_off"]), nbr_idx=_ptr(k["nbr_idx"]), is_bdy=_ptr(k["is_bdy"]),
            n_coll=_ptr(k["n_coll"]), T=_ptr(k["T"]), v_turb=_ptr(k["v_turb"]),
            n_spec=_ptr(k["n_spec"]), n_lev=sp.n_lev, n_lines=sp.n_lines, E=_ptr(k["E"]),
            g=_ptr(k["g"]), mass=sp.mass, up=_ptr(k["up"]), lo=_ptr(k["lo"]), A=_ptr(k["A"]),
            n_T=int(sp.T_grid.shape[0]), T_grid=_ptr(k["T_grid"]), K_down=_ptr(k["K_down"]),
            R=self.dirs.shape[0], Q=self.Q, dirs=_ptr(k["dirs"]), antipode=_ptr(k["anti"]),
            roots=_ptr(k["roots"]), weights=_ptr(k["weights"]), dshift_frac=dshift_frac,
            chi_min=chi_min, dtau_min=dtau_min, T_cmb=T_cmb, max_steps=max_steps)
        self.mp = C.byref(self.m)

    @property
    def n_lines(self):
        return self.model.species.n_lines

    def width(self, c):
        return _lib().or_width(self.mp, int(c))

    def trace(self, o, r):
        """Half-ray (o, r): dict of cells, nsub, ds, vpar (numpy arrays) and dead_end."""
        cap = self.m.max_steps
        cells = np.empty(cap, np.int32); nsub = np.empty(cap, np.int32)
        ds = np.empty(cap); vpar = np.empty(cap)
        ln = C.c_int64(0); de = C.c_int(0)
        rc = _lib().or_trace(self.mp, int(o), int(r), cap, _ptr(cells), _ptr(nsub), _ptr(ds),
                             _ptr(vpar), C.byref(ln), C.byref(de))
        if rc:
            raise RuntimeError(f"or_trace failed ({rc})")
        n = ln.value
        return dict(cells=cells[:n].copy(), nsub=nsub[:n].copy(), ds=ds[:n].copy(),
                    vpar=vpar[:n].copy(), dead_end=bool(de.value))

    def trace_all(self, origins=None):
        """All half-rays of the given origins: dict with off [n_orig*R+1] and flat
        cells, nsub, ds, vpar, plus dead [n_orig*R]."""
        if origins is None:
            origins = np.arange(self.model.n, dtype=np.int64)
        origins = np.ascontiguousarray(origins, np.int64)
        k = origins.shape[0] * self.dirs.shape[0]
        ln = np.zeros(k, np.int32)
        dead = np.zeros(k, np.uint8)
        L = _lib()
        if L.or_trace_all(self.mp, origins.shape[0], _ptr(origins), None, _ptr(ln), None, None, None, None,
                          _ptr(dead), self.nthreads):
            raise RuntimeError("or_trace_all failed")
        off = np.zeros(k + 1, np.int64)
        np.cumsum(ln, out=off[1:])
        tot = int(off[-1])
        cells = np.empty(tot, np.int32); nsub = np.empty(tot, np.int32)
        ds = np.empty(tot); vpar = np.empty(tot)
        if L.or_trace_all(self.mp, origins.shape[0], _ptr(origins), _ptr(off), _ptr(ln), _ptr(cells), _ptr(nsub),
                          _ptr(ds), _ptr(vpar), None, self.nthreads):
            raise RuntimeError("or_trace_all failed")
        return dict(off=off, cells=cells, nsub=nsub, ds=ds, vpar=vpar, dead=dead.astype(bool))

    def lte(self):
        pops = np.empty((self.model.n, self.model.species.n_lev))
        _lib().or_lte(self.mp, _ptr(pops))
        return pops

    def formal_solve(self, pops, origins=None, spectrum=False):
        """J, L, Jeff [n_orig][n_lines] (and Jnu [n_orig][n_lines][Q] if spectrum)."""
        pops = np.ascontiguousarray(pops, np.float64)
        if origins is None:
            origins = np.arange(self.model.n, dtype=np.int64)
        origins = np.ascontiguousarray(origins, np.int64)
        no, nl = origins.shape[0], self.n_lines
        J = np.empty((no, nl)); L = np.empty((no, nl)); E = np.empty((no, nl))
        Jnu = np.empty((no, nl, self.Q)) if spectrum else None
        rc = _lib().or_formal_solve(self.mp, _ptr(pops), no, _ptr(origins), _ptr(J), _ptr(L),
                                    _ptr(E), _ptr(Jnu), self.nthreads)
        if rc:
            raise RuntimeError(f"or_formal_solve failed ({rc})")
        return (J, L, E, Jnu) if spectrum else (J, L, E)

    def image(self, pops, ray, line, u_ch, origins=None):
        """Image along direction dirs[ray] (Sec. 3.5): intensity I [n_orig][n_ch] leaving
        the model along that direction on the ray pair through each origin, at channel
        frequencies nu_line (1 + u_ch/c) in the model's rest frame, and the origins'
        projections xy [n_orig][2] on the plane orthogonal to the direction."""
        pops = np.ascontiguousarray(pops, np.float64)
        if origins is None:
            origins = np.arange(self.model.n, dtype=np.int64)
        origins = np.ascontiguousarray(origins, np.int64)
        u = np.ascontiguousarray(u_ch, np.float64)
        I = np.empty((origins.shape[0], u.shape[0]))
        xy = np.empty((origins.shape[0], 2))
        rc = _lib().or_image(self.mp, _ptr(pops), int(ray), int(line), u.shape[0], _ptr(u),
                             origins.shape[0], _ptr(origins), _ptr(I), _ptr(xy), self.nthreads)
        if rc:
            raise RuntimeError(f"or_image failed ({rc})")
        return I, xy

    def formal_solve_band(self, pops, band, origins=None):
        """Formal solution with the band-diagonal ALO of bandwidth `band` (Sec. 3.4):
        J, L, [Jeff_0, ..., Jeff_band] (J_eff with the ALO's band 0..band), and the
        coupling coefficients M [n_orig][n_lines][R][band] of or_formal_solve_band."""
        pops = np.ascontiguousarray(pops, np.float64)
        if origins is None:
            origins = np.arange(self.model.n, dtype=np.int64)
        origins = np.ascontiguousarray(origins, np.int64)
        no, nl, R = origins.shape[0], self.n_lines, self.dirs.shape[0]
        J = np.empty((no, nl)); L = np.empty((no, nl)); E = np.empty((no, nl))
        Eb = np.empty((band, no, nl)); M = np.empty((no, nl, R, band))
        rc = _lib().or_formal_solve_band(self.mp, _ptr(pops), no, _ptr(origins), int(band), _ptr(J), _ptr(L),
                                         _ptr(E), _ptr(Eb), _ptr(M), self.nthreads)
        if rc:
            raise RuntimeError(f"or_formal_solve_band failed ({rc})")
        return J, L, [E] + [Eb[b] for b in range(band)], M

    def formal_solve_scattering(self, pops, chi_sca, tol=1e-10, max_iter=500, Jnu0=None):
        """Formal solution with isotropic, coherent scattering of opacity chi_sca [n]
        (Sec. 3.3, eq. 'GFE' with Psi+ = chi_sca J, Psi- = 0), the scattering source taken
        from the previous iteration's mean intensity as the section prescribes, starting
        from Jnu0 [n][n_lines][Q] (default: no scattered light) until the largest relative
        change of the per-bin mean intensity is below tol. Returns J, L, Jeff, Jnu and the
        list of changes."""
        pops = np.ascontiguousarray(pops, np.float64)
        m = self.model
        n, nl = m.n, self.n_lines
        chi_sca = np.ascontiguousarray(chi_sca, np.float64)
        orig = np.arange(n, dtype=np.int64)
        prev = np.zeros((n, nl, self.Q)) if Jnu0 is None else np.array(Jnu0, np.float64, copy=True)
        J = np.empty((n, nl)); L = np.empty((n, nl)); E = np.empty((n, nl))
        changes = []
        for it in range(max_iter):
            Jnu = np.empty((n, nl, self.Q))
            rc = _lib().or_formal_solve_sca(self.mp, _ptr(pops), n, _ptr(orig), _ptr(chi_sca), _ptr(prev), _ptr(J),
                                            _ptr(L), _ptr(E), _ptr(Jnu), self.nthreads)
            if rc:
                raise RuntimeError(f"or_formal_solve_sca failed ({rc})")
            ch = float(np.max(np.abs(Jnu - prev) / Jnu))
            changes.append(ch)
            prev = Jnu
            if ch < tol:
                break
        return J, L, E, prev, changes

    def band_geometry(self, band, origins=None):
        """Cells (ca, cb) and weight w of the j-th expanded point of every half-ray,
        [n_orig][R][band] (ca = cb = -1 where the half is shorter)."""
        if origins is None:
            origins = np.arange(self.model.n, dtype=np.int64)
        origins = np.ascontiguousarray(origins, np.int64)
        R = self.dirs.shape[0]
        shape = (origins.shape[0], R, band)
        ca = np.empty(shape, np.int32); cb = np.empty(shape, np.int32); w = np.empty(shape)
        if _lib().or_band_geometry(self.mp, origins.shape[0], _ptr(origins), int(band), _ptr(ca), _ptr(cb), _ptr(w)):
            raise RuntimeError("or_band_geometry failed")
        return ca, cb, w

    def cell_generator(self, c, oml, Jeff_c):
        """Rate generator of cell c (eq. 'ourALI'), G[i][j] = rate j -> i."""
        lev = self.model.species.n_lev
        G = np.empty((lev, lev))
        if _lib().or_cell_generator(self.mp, int(c), _ptr(np.ascontiguousarray(oml, np.float64)),
                                    _ptr(np.ascontiguousarray(Jeff_c, np.float64)), _ptr(G)):
            raise RuntimeError("or_cell_generator failed")
        return G

    def band_system(self, L, Jeff, M, geom, b, pops_old):
        """The rate equations of all cells with the ALO of bandwidth b (eq. 'ourALI' with
        the operator of eq. 'ALO'), as one sparse linear system A n = rhs over all cells
        and levels. Per cell o and line l = (u -> lo), the band points of every half-ray
        contribute A_ul M n_u at the point, n_u interpolated between the point's cells
        (ca, cb) with weight w: the part on the origin itself (ca = o) lowers the factor
        1 - L of the spontaneous rate, the other cells enter as couplings (+ to the balance
        of u, - to that of lo). The last balance equation of each cell is replaced by
        sum_i n_i = n_spec. Returns (A as scipy CSR, rhs)."""
        import scipy.sparse as sps
        m, sp = self.model, self.model.species
        n, lev, nl = m.n, sp.n_lev, sp.n_lines
        ca, cb, w = geom
        rows, cols, vals = [], [], []
        rhs = np.zeros(n * lev)
        for o in range(n):
            oml = 1.0 - L[o]
            coup = []                       # (line, cell, weight x M)
            for l in range(nl):
                for r in range(ca.shape[1]):
                    for j in range(b):
                        Mv = M[o, l, r, j]
                        if ca[o, r, j] < 0 or Mv == 0.0:
                            continue
                        for cell, wt in ((cb[o, r, j], w[o, r, j]), (ca[o, r, j], 1.0 - w[o, r, j])):
                            if wt == 0.0:
                                continue
                            if cell == o:
                                oml[l] -= wt * Mv
                            else:
                                coup.append((l, cell, wt * Mv))
            G = self.cell_generator(o, oml, Jeff[o])
            for i in range(lev - 1):
                for j in range(lev):
                    if G[i, j] != 0.0:
                        rows.append(o * lev + i); cols.append(o * lev + j); vals.append(G[i, j])
            for j in range(lev):
                rows.append(o * lev + lev - 1); cols.append(o * lev + j); vals.append(1.0)
            rhs[o * lev + lev - 1] = m.n_spec[o]
            for l, cell, cf in coup:
                u, lo = int(sp.up[l]), int(sp.lo[l])
                a = sp.A[l] * cf
                if u < lev - 1:
                    rows.append(o * lev + u); cols.append(cell * lev + u); vals.append(a)
                if lo < lev - 1:
                    rows.append(o * lev + lo); cols.append(cell * lev + u); vals.append(-a)
        A = sps.csr_matrix((vals, (rows, cols)), shape=(n * lev, n * lev))
        A.sum_duplicates()
        return A, rhs

    def solve_band(self, L, Jeff, M, geom, b, pops_old):
        """Solution of band_system by sparse LU (scipy's SuperLU), with the unknowns
        scaled by the old populations (floored at 1e-20 of the cell's species density) so
        that levels of very different size are resolved alike."""
        import scipy.sparse as sps
        import scipy.sparse.linalg as spl
        A, rhs = self.band_system(L, Jeff, M, geom, b, pops_old)
        ns = self.model.n_spec
        s = np.maximum(np.asarray(pops_old, np.float64), 1e-20 * ns[:, None]).ravel()
        x = spl.spsolve((A @ sps.diags(s)).tocsc(), rhs)
        return (x * s).reshape(pops_old.shape)

    def stateq_band(self, J, L, Jeffs, M, geom, band, pops_old):
        """Statistical equilibrium with the band-diagonal ALO and its validity check
        (Sec. 6.1): the system of bandwidth b is solved; if any population comes out
        negative or non-finite it is solved again with bandwidth b - 1, down to the
        diagonal ALO, whose own check re-solves single cells without the ALO.
        Returns (pops, bandwidth used, fallback cells of the diagonal stage)."""
        for b in range(band, 0, -1):
            pops = self.solve_band(L, Jeffs[b], M, geom, b, pops_old)
            if np.all(np.isfinite(pops)) and np.all(pops >= 0.0):
                return pops, b, 0
        pops, nf = self.stateq(J, L, Jeffs[0])
        return pops, 0, nf

    def ali_band(self, band, pops=None, tol=1e-6, max_iter=200, ng_period=0, grow_limit=3):
        """ALI with the band-diagonal ALO (formal solve -> band statistical equilibrium ->
        convergence), Ng as in or_ali. The bandwidth in use starts at `band` and only
        decreases (Sec. 6.1, "reduce the bandwidth if required"; Reading: a reduction
        holds for the rest of the ALI): when the validity check of stateq_band had to
        reduce it, and when the max relative change has grown in `grow_limit` consecutive
        iterations (a diverging ALI), by one. Returns (pops, changes, converged, bandwidth
        used per iteration)."""
        pops = self.lte() if pops is None else np.array(pops, np.float64, copy=True)
        geom = self.band_geometry(band) if band > 0 else None
        ns = self.model.n_spec[:, None]
        hist, changes, used = [], [], []
        nh, grow, b_cur = 0, 0, band
        conv = False
        for it in range(max_iter):
            if b_cur > 0:
                J, L, Jeffs, M = self.formal_solve_band(pops, b_cur)
                g = tuple(x[..., :b_cur] for x in geom)
                new, b_used, nf = self.stateq_band(J, L, Jeffs, M, g, b_cur, pops)
            else:
                J, L, E = self.formal_solve(pops)
                new, nf = self.stateq(J, L, E)
                b_used = 0
            ch = self.max_rel_change(pops, new)
            grow = grow + 1 if changes and ch > changes[-1] else 0
            changes.append(ch); used.append(b_used)
            b_cur = min(b_cur, b_used)
            if grow >= grow_limit and b_cur > 0:
                b_cur -= 1
                grow = 0
            pops = new
            if ch < tol:
                conv = True
                break
            if ng_period > 0:
                hist.insert(0, pops / ns)
                hist = hist[:4]
                nh = min(nh + 1, 4)
                if nh == 4 and (it + 1) % ng_period == 0:
                    try:
                        x = ng(*[np.ascontiguousarray(h) for h in hist])
                        if np.all(x >= 0.0):
                            pops = x * ns
                    except RuntimeError:
                        pass
                    nh = 0
        return pops, np.array(changes), conv, used

    def stateq(self, J, L, Jeff):
        out = np.empty((self.model.n, self.model.species.n_lev))
        nf = C.c_int64(0)
        rc = _lib().or_stateq(self.mp, _ptr(np.ascontiguousarray(J)), _ptr(np.ascontiguousarray(L)),
                              _ptr(np.ascontiguousarray(Jeff)), _ptr(out), C.byref(nf))
        if rc:
            raise RuntimeError("or_stateq failed")
        return out, nf.value

    def max_rel_change(self, old, new):
        return _lib().or_max_rel_change(self.mp, _ptr(np.ascontiguousarray(old)),
                                        _ptr(np.ascontiguousarray(new)))

    def ali(self, pops=None, tol=1e-6, max_iter=200, ng_period=0):
        """Run the ALI; returns (pops, changes, converged)."""
        pops = self.lte() if pops is None else np.array(pops, np.float64, copy=True)
        ch = np.zeros(max_iter)
        conv = C.c_int(0)
        it = _lib().or_ali(self.mp, _ptr(pops), tol, max_iter, ng_period, _ptr(ch),
                           C.byref(conv), self.nthreads)
        if it < 0:
            raise RuntimeError(f"or_ali failed ({it})")
        return pops, ch[:it].copy(), bool(conv.value)


def ng(x0, x1, x2, x3):
    out = np.empty_like(x0)
    rc = _lib().or_ng(x0.size, _ptr(x0), _ptr(x1), _ptr(x2), _ptr(x3), _ptr(out))
    if rc:
        raise RuntimeError("singular Ng system")
    return out


def feautrier(dtau, S, I0, IK, ko):
    """u and Lambda*_oo at index ko of the discretised second-order transfer equation."""
    dtau = np.ascontiguousarray(dtau, np.float64); S = np.ascontiguousarray(S, np.float64)
    K = S.shape[0]
    work = np.empty(5 * K)
    u = C.c_double(0); lam = C.c_double(0)
    _lib().or_feautrier(K, int(ko), _ptr(dtau), _ptr(S), float(I0), float(IK), C.byref(u),
                        C.byref(lam), _ptr(work))
    return u.value, lam.value


def feautrier_row(dtau, ko, band=None):
    """Entries |k - ko| <= band (default: the whole row) of row ko of the inverse of the
    discretised second-order transfer operator: the weights of the sources at the points
    in u at ko. Entries outside the band are NaN."""
    dtau = np.ascontiguousarray(dtau, np.float64)
    K = dtau.shape[0] + 1
    x = np.full(K, np.nan); work = np.empty(6 * K)
    if _lib().or_feautrier_band(K, int(ko), int(K if band is None else band), _ptr(dtau), _ptr(x), _ptr(work)):
        raise RuntimeError("or_feautrier_band needs at least two points")
    return x


def first_order(dtau, S, I0):
    """Outward intensity of dI/dtau = S - I over points with increments dtau, S linear in
    tau between points (Olson & Kunasz 1987), entering with I0."""
    dtau = np.ascontiguousarray(dtau, np.float64); S = np.ascontiguousarray(S, np.float64)
    return _lib().or_first_order(S.shape[0], _ptr(dtau), _ptr(S), float(I0))
