"""ctypes binding of libmagritte_gb300 (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; this module only converts
numpy arrays and device pointers into the C ABI declared in include/magritte_gb300.h.
There is no fallback: if the library cannot be loaded, import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MG_OK = 0
MG_ERR_ARG, MG_ERR_STATE, MG_ERR_CUDA, MG_ERR_OOM = -1, -2, -3, -4
MG_ERR_NOT_CONVERGED, MG_ERR_NUMERIC, MG_ERR_CAPACITY = -5, -6, -7
MG_WARN_DEAD_END_RAYS, MG_WARN_NEG_POP_FALLBACK, MG_WARN_NEG_OPACITY = 1, 2, 3
MG_FP64, MG_MIXED = 0, 1
MG_GEOM_3D, MG_GEOM_SPHERICAL_1D = 0, 1
MG_INIT_LTE, MG_INIT_GIVEN, MG_INIT_MLP = 0, 1, 2


class mg_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("ng_period", C.c_int32), ("dshift_frac", C.c_double),
                ("chi_min", C.c_double), ("dtau_min", C.c_double), ("T_cmb", C.c_double),
                ("line_cut", C.c_double), ("max_steps", C.c_int64), ("profile", C.c_int32),
                ("spectrum", C.c_int32), ("pad", C.c_int32), ("tau_fp64", C.c_double),
                ("alo_band", C.c_int32), ("pad2", C.c_int32)]


class mg_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("pad", C.c_int32),
                ("seed", C.c_uint64)]


class mg_train_report(C.Structure):
    _fields_ = [("first_loss", C.c_double), ("last_loss", C.c_double), ("steps", C.c_int64),
                ("seconds", C.c_double)]


class mg_ray_stats(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("n_elements", C.c_int64), ("n_expanded", C.c_int64),
                ("max_pair_len", C.c_int64), ("n_dead_end", C.c_int64), ("mean_pair_len", C.c_double)]


class mg_ali_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("ng_steps", C.c_int32), ("converged", C.c_int32),
                ("alo_band", C.c_int32), ("last_change", C.c_double), ("n_fallback", C.c_int64),
                ("seconds", C.c_double)]


class MagritteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_P = C.c_void_p
_SIGS = {
    "mg_default_options": (None, [_P]),
    "mg_create": (C.c_int, [_P, _P]),
    "mg_destroy": (C.c_int, [_P]),
    "mg_last_error": (C.c_char_p, [_P]),
    "mg_set_stream": (C.c_int, [_P, _P]),
    "mg_set_mesh": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int32]),
    "mg_set_model": (C.c_int, [_P, _P, _P, _P, _P]),
    "mg_set_species": (C.c_int, [_P, C.c_int32, _P, _P, C.c_double, C.c_int32, _P, _P, _P, C.c_int32, _P, _P]),
    "mg_set_directions": (C.c_int, [_P, C.c_int32]),
    "mg_set_directions_custom": (C.c_int, [_P, C.c_int32, _P]),
    "mg_get_directions": (C.c_int, [_P, _P, _P, _P]),
    "mg_set_quadrature": (C.c_int, [_P, C.c_int32]),
    "mg_get_quadrature": (C.c_int, [_P, _P, _P]),
    "mg_trace_rays": (C.c_int, [_P, _P]),
    "mg_get_ray": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P, _P, C.c_int64, _P]),
    "mg_init_populations": (C.c_int, [_P, C.c_int32]),
    "mg_set_populations": (C.c_int, [_P, _P]),
    "mg_get_populations": (C.c_int, [_P, _P]),
    "mg_set_populations_dev": (C.c_int, [_P, _P]),
    "mg_get_populations_dev": (C.c_int, [_P, _P]),
    "mg_formal_solve": (C.c_int, [_P]),
    "mg_get_radiation": (C.c_int, [_P, _P, _P, _P]),
    "mg_get_radiation_dev": (C.c_int, [_P, _P, _P, _P]),
    "mg_set_radiation": (C.c_int, [_P, _P, _P, _P]),
    "mg_get_spectrum": (C.c_int, [_P, _P]),
    "mg_image": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]),
    "mg_image_dev": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]),
    "mg_update_populations": (C.c_int, [_P, _P]),
    "mg_update_populations_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "mg_iterate": (C.c_int, [_P, _P]),
    "mg_kernel_times": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "mg_reset_kernel_times": (C.c_int, [_P]),
    "mg_work_counts": (C.c_int, [_P, _P, _P]),
    "mg_executed_work": (C.c_int, [_P, _P]),
    "mg_measure_pipe_rates": (C.c_int, [C.c_int32, _P]),
    "mg_autotune": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_status_counts": (C.c_int, [_P, _P, _P]),
    "mg_band_status": (C.c_int, [_P, _P, _P]),
    "mg_set_scattering": (C.c_int, [_P, _P, C.c_double, C.c_int32]),
    "mg_scattering_status": (C.c_int, [_P, _P, _P]),
    "mg_get_band_terms": (C.c_int, [_P, _P, _P, _P]),
    "mg_promoted_cells": (C.c_int, [_P, _P]),
    "mg_mlp_create": (C.c_int, [_P, C.c_int32, C.c_uint64, C.c_int32]),
    "mg_mlp_destroy": (C.c_int, [_P]),
    "mg_mlp_last_error": (C.c_char_p, [_P]),
    "mg_mlp_param_count": (C.c_int, [_P, _P]),
    "mg_mlp_set_params": (C.c_int, [_P, _P, C.c_int64]),
    "mg_mlp_get_params": (C.c_int, [_P, _P, C.c_int64]),
    "mg_mlp_set_normalisation": (C.c_int, [_P, _P, _P]),
    "mg_mlp_forward": (C.c_int, [_P, C.c_int64, _P, _P]),
    "mg_mlp_loss_grad": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "mg_mlp_train": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    "mg_features": (C.c_int, [_P, _P]),
    "mg_attach_mlp": (C.c_int, [_P, _P]),
    "mg_mlp_save": (C.c_int, [_P, C.c_char_p]),
    "mg_mlp_load": (C.c_int, [_P, C.c_char_p, C.c_int32]),
    "mg_init_populations_mlp": (C.c_int, [_P, _P]),
    "mg_batch_create": (C.c_int, [_P, C.c_int32, _P]),
    "mg_batch_destroy": (C.c_int, [_P]),
    "mg_batch_last_error": (C.c_char_p, [_P]),
    "mg_batch_formal_solve": (C.c_int, [_P]),
    "mg_batch_iterate": (C.c_int, [_P, _P]),
    "mg_batch_set_variant": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "mg_batch_autotune": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "mg_batch_work_counts": (C.c_int, [_P, _P, _P]),
    "mg_set_variant": (C.c_int, [_P, C.c_int32]),
}

_LIB = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads the shared library (building it first if needed) and declares signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libmagritte_gb300 not built: {path}")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def declared_symbols():
    return list(_SIGS)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return C.c_void_p(a)
    return C.c_void_p(a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def default_options(**kw):
    o = mg_options()
    load().mg_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def measure_pipe_rates(device=0):
    """Measured FP32 pipe throughput on a device: dict with ffma, ffma2 (flops/s), ex2,
    rcp (results/s)."""
    r = np.zeros(4)
    rc = load().mg_measure_pipe_rates(int(device), _ptr(r))
    if rc != MG_OK:
        raise MagritteError(rc, "mg_measure_pipe_rates failed")
    return dict(ffma=float(r[0]), ffma2=float(r[1]), ex2=float(r[2]), rcp=float(r[3]))


class Context:
    """Owns one mg_ctx. Methods mirror the C functions of the same name."""

    def __init__(self, **options):
        self.lib = load()
        self.opt = default_options(**options)
        h = C.c_void_p()
        rc = self.lib.mg_create(C.byref(h), C.byref(self.opt))
        if rc != MG_OK:
            raise MagritteError(rc, "mg_create failed")
        self.h = h
        self.n = 0
        self.n_lev = 0
        self.n_lines = 0
        self.Q = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what, warn_ok=True):
        if rc < 0 or (rc > 0 and not warn_ok):
            msg = self.lib.mg_last_error(self.h)
            raise MagritteError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    # ---- set-up
    def set_stream(self, stream_ptr):
        return self._chk(self.lib.mg_set_stream(self.h, C.c_void_p(stream_ptr) if stream_ptr else None), "mg_set_stream")

    def set_mesh(self, pos, vel, nbr_off, nbr_idx, is_bdy, geometry=MG_GEOM_3D):
        pos, vel = _c(pos, np.float64), _c(vel, np.float64)
        off, idx, bdy = _c(nbr_off, np.int64), _c(nbr_idx, np.int32), _c(is_bdy, np.uint8)
        n = pos.shape[0]
        self._chk(self.lib.mg_set_mesh(self.h, n, _ptr(pos), _ptr(vel), _ptr(off), _ptr(idx), _ptr(bdy),
                                       int(geometry)), "mg_set_mesh")
        self.n = n

    def set_model(self, n_coll, T, v_turb, n_species):
        a = [_c(x, np.float64) for x in (n_coll, T, v_turb, n_species)]
        self._chk(self.lib.mg_set_model(self.h, *[_ptr(x) for x in a]), "mg_set_model")

    def set_species(self, E, g, mass, up, lo, A, T_grid, K_down):
        E, g, A = _c(E, np.float64), _c(g, np.float64), _c(A, np.float64)
        up, lo = _c(up, np.int32), _c(lo, np.int32)
        Tg, K = _c(T_grid, np.float64), _c(K_down, np.float64)
        self._chk(self.lib.mg_set_species(self.h, E.shape[0], _ptr(E), _ptr(g), float(mass), A.shape[0],
                                          _ptr(up), _ptr(lo), _ptr(A), Tg.shape[0], _ptr(Tg), _ptr(K)),
                  "mg_set_species")
        self.n_lev, self.n_lines = E.shape[0], A.shape[0]

    def set_directions(self, nside):
        self._chk(self.lib.mg_set_directions(self.h, int(nside)), "mg_set_directions")

    def set_directions_custom(self, dirs):
        d = _c(dirs, np.float64)
        self._chk(self.lib.mg_set_directions_custom(self.h, d.shape[0], _ptr(d)), "mg_set_directions_custom")

    def get_directions(self):
        R = C.c_int32(0)
        self._chk(self.lib.mg_get_directions(self.h, C.byref(R), None, None), "mg_get_directions")
        d = np.empty((R.value, 3)); a = np.empty(R.value, np.int32)
        self._chk(self.lib.mg_get_directions(self.h, None, _ptr(d), _ptr(a)), "mg_get_directions")
        return d, a

    def set_quadrature(self, n_q):
        self._chk(self.lib.mg_set_quadrature(self.h, int(n_q)), "mg_set_quadrature")
        self.Q = int(n_q)

    def get_quadrature(self):
        r = np.empty(self.Q); w = np.empty(self.Q)
        self._chk(self.lib.mg_get_quadrature(self.h, _ptr(r), _ptr(w)), "mg_get_quadrature")
        return r, w

    def trace_rays(self):
        st = mg_ray_stats()
        rc = self._chk(self.lib.mg_trace_rays(self.h, C.byref(st)), "mg_trace_rays")
        return {k: getattr(st, k) for k, _ in st._fields_}, rc

    def get_ray(self, point, ray, cap=1 << 16):
        cells = np.empty(cap, np.int32); nsub = np.empty(cap, np.int32)
        ds = np.empty(cap); vpar = np.empty(cap); ln = C.c_int64(0)
        self._chk(self.lib.mg_get_ray(self.h, int(point), int(ray), _ptr(cells), _ptr(nsub), _ptr(ds), _ptr(vpar),
                                      cap, C.byref(ln)), "mg_get_ray")
        n = ln.value
        return dict(cells=cells[:n].copy(), nsub=nsub[:n].copy(), ds=ds[:n].copy(), vpar=vpar[:n].copy())

    # ---- populations and solves
    def init_populations(self, mode=MG_INIT_LTE):
        self._chk(self.lib.mg_init_populations(self.h, int(mode)), "mg_init_populations")

    def set_populations(self, pops):
        p = _c(pops, np.float64)
        self._chk(self.lib.mg_set_populations(self.h, _ptr(p)), "mg_set_populations")

    def get_populations(self, out=None):
        p = np.empty((self.n, self.n_lev)) if out is None else out
        self._chk(self.lib.mg_get_populations(self.h, _ptr(p)), "mg_get_populations")
        return p

    def set_populations_dev(self, dev_ptr):
        self._chk(self.lib.mg_set_populations_dev(self.h, C.c_void_p(dev_ptr)), "mg_set_populations_dev")

    def get_populations_dev(self, dev_ptr):
        self._chk(self.lib.mg_get_populations_dev(self.h, C.c_void_p(dev_ptr)), "mg_get_populations_dev")

    def formal_solve(self):
        self._chk(self.lib.mg_formal_solve(self.h), "mg_formal_solve")

    def get_radiation(self):
        J = np.empty((self.n, self.n_lines)); L = np.empty_like(J); E = np.empty_like(J)
        self._chk(self.lib.mg_get_radiation(self.h, _ptr(J), _ptr(L), _ptr(E)), "mg_get_radiation")
        return J, L, E

    def set_radiation(self, J, L, Jeff):
        """Replaces the radiation field read by update_populations (mg_set_radiation)."""
        J, L, E = _c(J, np.float64), _c(L, np.float64), _c(Jeff, np.float64)
        self._chk(self.lib.mg_set_radiation(self.h, _ptr(J), _ptr(L), _ptr(E)), "mg_set_radiation")

    def get_spectrum(self):
        out = np.empty((self.n, self.n_lines, self.Q))
        self._chk(self.lib.mg_get_spectrum(self.h, _ptr(out)), "mg_get_spectrum")
        return out

    def image(self, ray, line, u_ch):
        """Image along dirs[ray]: intensity I [n][n_ch] at channel offsets u_ch (m/s) of
        line `line`, and sky-plane coordinates xy [n][2]."""
        u = _c(u_ch, np.float64)
        I = np.empty((self.n, u.shape[0])); xy = np.empty((self.n, 2))
        self._chk(self.lib.mg_image(self.h, int(ray), int(line), u.shape[0], _ptr(u), _ptr(I), _ptr(xy)), "mg_image")
        return I, xy

    def image_dev(self, ray, line, u_ch, d_I, d_xy=None):
        """mg_image into device buffers (integer device addresses)."""
        u = _c(u_ch, np.float64)
        self._chk(self.lib.mg_image_dev(self.h, int(ray), int(line), u.shape[0], _ptr(u), _ptr(d_I),
                                        _ptr(d_xy)), "mg_image_dev")

    def update_populations(self):
        ch = C.c_double(0)
        rc = self._chk(self.lib.mg_update_populations(self.h, C.byref(ch)), "mg_update_populations")
        return ch.value, rc

    def update_populations_noalloc(self, d_old, d_new):
        """Allocation-free statistical-equilibrium update between caller-owned device
        buffers (see mg_update_populations_noalloc)."""
        ch = C.c_double(0); nf = C.c_int64(0)
        rc = self._chk(self.lib.mg_update_populations_noalloc(self.h, C.c_void_p(d_old), C.c_void_p(d_new),
                                                              C.byref(ch), C.byref(nf)),
                       "mg_update_populations_noalloc")
        return ch.value, nf.value, rc

    def iterate(self, allow_not_converged=False):
        rep = mg_ali_report()
        rc = self.lib.mg_iterate(self.h, C.byref(rep))
        if rc < 0 and not (allow_not_converged and rc == MG_ERR_NOT_CONVERGED):
            self._chk(rc, "mg_iterate")
        return {k: getattr(rep, k) for k, _ in rep._fields_ if k != "pad"}, rc

    def kernel_times(self):
        cap = 64
        names = (C.c_char_p * cap)(); ms = np.zeros(cap); la = np.zeros(cap, np.int64); cnt = C.c_int32(0)
        self._chk(self.lib.mg_kernel_times(self.h, cap, names, _ptr(ms), _ptr(la), C.byref(cnt)), "mg_kernel_times")
        return {names[i].decode(): (float(ms[i]), int(la[i])) for i in range(min(cnt.value, cap))}

    def reset_kernel_times(self):
        self._chk(self.lib.mg_reset_kernel_times(self.h), "mg_reset_kernel_times")

    def promoted_cells(self):
        c = C.c_int64(0)
        self._chk(self.lib.mg_promoted_cells(self.h, C.byref(c)), "mg_promoted_cells")
        return c.value

    def status_counts(self):
        f = C.c_int64(0); n = C.c_int64(0)
        self._chk(self.lib.mg_status_counts(self.h, C.byref(f), C.byref(n)), "mg_status_counts")
        return f.value, n.value

    def set_scattering(self, chi_sca, tol=1e-8, max_iter=100):
        """Isotropic coherent scattering of opacity chi_sca [n] (None switches it off)."""
        x = None if chi_sca is None else _c(chi_sca, np.float64)
        self._chk(self.lib.mg_set_scattering(self.h, _ptr(x), float(tol), int(max_iter)), "mg_set_scattering")

    def scattering_status(self):
        """(passes, final relative change) of the last formal solve's scattering iteration."""
        it = C.c_int32(0); ch = C.c_double(0)
        self._chk(self.lib.mg_scattering_status(self.h, C.byref(it), C.byref(ch)), "mg_scattering_status")
        return it.value, ch.value

    def band_status(self):
        """(bandwidth in use, GMRES iterations since populations were set)."""
        b = C.c_int32(0); it = C.c_int64(0)
        self._chk(self.lib.mg_band_status(self.h, C.byref(b), C.byref(it)), "mg_band_status")
        return b.value, it.value

    def get_band_terms(self):
        """J_eff of bandwidths 1..B [B][n][n_lines] and coupling terms M [n][n_lines][R][B]
        of the last formal solve."""
        B = C.c_int32(0)
        self._chk(self.lib.mg_get_band_terms(self.h, C.byref(B), None, None), "mg_get_band_terms")
        R = self.get_directions()[0].shape[0]
        Jb = np.empty((B.value, self.n, self.n_lines)); M = np.empty((self.n, self.n_lines, R, B.value))
        self._chk(self.lib.mg_get_band_terms(self.h, C.byref(B), _ptr(Jb), _ptr(M)), "mg_get_band_terms")
        return Jb, M

    def features(self):
        out = np.empty((self.n, 4), np.float32)
        self._chk(self.lib.mg_features(self.h, _ptr(out)), "mg_features")
        return out

    def init_populations_mlp(self, mlp):
        self._chk(self.lib.mg_init_populations_mlp(self.h, mlp.h), "mg_init_populations_mlp")

    def attach_mlp(self, mlp):
        """Attaches a network for init_populations(MG_INIT_MLP) (None detaches); the
        context keeps a reference so that the network outlives the attachment."""
        self._chk(self.lib.mg_attach_mlp(self.h, mlp.h if mlp is not None else None), "mg_attach_mlp")
        self._mlp = mlp

    def autotune(self, reps=2):
        v = C.c_int32(0); ms = C.c_double(0); nt = C.c_int32(0)
        self._chk(self.lib.mg_autotune(self.h, int(reps), C.byref(v), C.byref(ms), C.byref(nt)), "mg_autotune")
        return v.value, ms.value, nt.value

    def set_variant(self, v):
        self._chk(self.lib.mg_set_variant(self.h, int(v)), "mg_set_variant")

    def work_counts(self):
        s = C.c_int64(0); u = C.c_int64(0)
        self._chk(self.lib.mg_work_counts(self.h, C.byref(s), C.byref(u)), "mg_work_counts")
        return s.value, u.value

    def executed_work(self):
        """Point-bin updates the warp kernel executed since reset_kernel_times (profiling)."""
        u = C.c_int64(0)
        self._chk(self.lib.mg_executed_work(self.h, C.byref(u)), "mg_executed_work")
        return u.value

    # ---- convenience: load a synthetic model
    def load_model(self, m, nside=None, dirs=None, n_q=None):
        """Copies a synthetic.Model into the context (mesh, fields, species, directions,
        quadrature)."""
        sp = m.species
        self.set_mesh(m.pos, m.vel, m.nbr_off, m.nbr_idx, m.is_bdy, m.geometry)
        self.set_species(sp.E, sp.g, sp.mass, sp.up, sp.lo, sp.A, sp.T_grid, sp.K_down)
        self.set_model(m.n_coll, m.T, m.v_turb, m.n_spec)
        d = dirs if dirs is not None else m.dirs
        if d is not None:
            self.set_directions_custom(d)
        else:
            self.set_directions(nside if nside is not None else m.nside)
        self.set_quadrature(n_q if n_q is not None else m.n_q)


class Batch:
    """Owns one mg_batch over existing Contexts (which must outlive it)."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = C.c_void_p()
        rc = self.lib.mg_batch_create(C.byref(h), len(self.contexts), arr)
        if rc != MG_OK:
            msg = self.lib.mg_last_error(self.contexts[0].h)
            raise MagritteError(rc, f"mg_batch_create: {msg.decode() if msg else ''}")
        self.h = h

    def _chk(self, rc, what):
        if rc < 0:
            msg = self.lib.mg_batch_last_error(self.h)
            raise MagritteError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def formal_solve(self):
        self._chk(self.lib.mg_batch_formal_solve(self.h), "mg_batch_formal_solve")

    def iterate(self, allow_not_converged=False):
        reps = (mg_ali_report * len(self.contexts))()
        rc = self.lib.mg_batch_iterate(self.h, reps)
        if rc < 0 and not (allow_not_converged and rc == MG_ERR_NOT_CONVERGED):
            self._chk(rc, "mg_batch_iterate")
        return [{k: getattr(r, k) for k, _ in r._fields_ if k != "pad"} for r in reps], rc

    def set_variant(self, variant, sorted_queue=True):
        self._chk(self.lib.mg_batch_set_variant(self.h, int(variant), 1 if sorted_queue else 0),
                  "mg_batch_set_variant")

    def autotune(self, reps=2):
        v = C.c_int32(0); s = C.c_int32(0); ms = C.c_double(0)
        self._chk(self.lib.mg_batch_autotune(self.h, int(reps), C.byref(v), C.byref(s), C.byref(ms)), "mg_batch_autotune")
        return v.value, s.value, ms.value

    def work_counts(self):
        s = C.c_int64(0); u = C.c_int64(0)
        self._chk(self.lib.mg_batch_work_counts(self.h, C.byref(s), C.byref(u)), "mg_batch_work_counts")
        return s.value, u.value


MLP_IN = 4   # network inputs per cell (mg_features)


def _rows(X, width, what):
    X = _c(X, np.float32)
    if X.ndim != 2 or X.shape[1] != width:
        raise ValueError(f"{what}: expected rows of {width} values, got shape {X.shape}")
    return X


class MLP:
    """Owns one mg_mlp (learned initial populations)."""

    def __init__(self, n_out, seed=0, device=0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.mg_mlp_create(C.byref(h), int(n_out), int(seed), int(device))
        if rc != MG_OK:
            raise MagritteError(rc, "mg_mlp_create failed")
        self.h = h
        self.n_out = int(n_out)
        c = C.c_int64(0)
        self.lib.mg_mlp_param_count(self.h, C.byref(c))
        self.n_params = c.value

    def _chk(self, rc, what):
        if rc < 0:
            msg = self.lib.mg_mlp_last_error(self.h)
            raise MagritteError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        t = np.empty(self.n_params, np.float32)
        self._chk(self.lib.mg_mlp_get_params(self.h, _ptr(t), self.n_params), "mg_mlp_get_params")
        return t

    def set_params(self, theta):
        t = _c(theta, np.float32)
        self._chk(self.lib.mg_mlp_set_params(self.h, _ptr(t), t.size), "mg_mlp_set_params")

    def save(self, path):
        self._chk(self.lib.mg_mlp_save(self.h, str(path).encode()), "mg_mlp_save")

    @classmethod
    def load(cls, path, device=0):
        """A network read from a file written by save()."""
        self = cls.__new__(cls)
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.mg_mlp_load(C.byref(h), str(path).encode(), int(device))
        if rc != MG_OK:
            raise MagritteError(rc, f"mg_mlp_load: cannot read a network from {path}")
        self.h = h
        c = C.c_int64(0)
        self.lib.mg_mlp_param_count(self.h, C.byref(c))
        self.n_params = c.value
        self.n_out = (self.n_params - (MLP_IN * 128 + 128 + 2 * (128 * 128 + 128))) // 129
        return self

    def set_normalisation(self, mean, std):
        m, s = _c(mean, np.float32), _c(std, np.float32)
        if m.size != MLP_IN or s.size != MLP_IN:
            raise ValueError(f"set_normalisation: expected {MLP_IN} means and standard deviations")
        self.mean, self.std = m, s
        self._chk(self.lib.mg_mlp_set_normalisation(self.h, _ptr(m), _ptr(s)), "mg_mlp_set_normalisation")

    def forward(self, X):
        X = _rows(X, MLP_IN, "forward")
        out = np.empty((X.shape[0], self.n_out), np.float32)
        self._chk(self.lib.mg_mlp_forward(self.h, X.shape[0], _ptr(X), _ptr(out)), "mg_mlp_forward")
        return out

    def loss_grad(self, X, Y):
        X, Y = _rows(X, MLP_IN, "loss_grad"), _rows(Y, self.n_out, "loss_grad")
        loss = C.c_double(0)
        g = np.empty(self.n_params, np.float32)
        self._chk(self.lib.mg_mlp_loss_grad(self.h, X.shape[0], _ptr(X), _ptr(Y), C.byref(loss), _ptr(g)),
                  "mg_mlp_loss_grad")
        return loss.value, g

    def train(self, X, Y, epochs=10, batch=4096, lr=1e-3, seed=0):
        X, Y = _rows(X, MLP_IN, "train"), _rows(Y, self.n_out, "train")
        o = mg_train_opts(epochs=epochs, batch=batch, lr=lr, seed=seed)
        r = mg_train_report()
        self._chk(self.lib.mg_mlp_train(self.h, X.shape[0], _ptr(X), _ptr(Y), C.byref(o), C.byref(r)), "mg_mlp_train")
        return {k: getattr(r, k) for k, _ in r._fields_}

