"""Thin ctypes binding of libhfx.so (include/hfx.h), same entry-point names.

Argument marshalling only: every step of the exchange-matrix build runs in the
CUDA library.  There is no CPU fallback: if the library is missing or cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

HFX_OK = 0
HFX_EINVAL = -1
HFX_ENOTHERM = -2
HFX_ENONFINITE = -3
HFX_EMISSING = -4
HFX_EDEVICE = -5
HFX_ETIMEOUT = -6
HFX_ENOMEM = -7
HFX_ENOTSPARSE = -8
HFX_EUNSUPPORTED = -9

HFX_PREC_FP64 = 0
HFX_PREC_SLICED = 1
HFX_SPARSE_AUTO, HFX_SPARSE_ON, HFX_SPARSE_OFF = 0, 1, 2
HFX_LAYOUT_DENSE, HFX_LAYOUT_TRANSFORMED, HFX_LAYOUT_TRANSFORMED_ONSITE = 0, 1, 2

EXPORTS = (
    "hfx_default_options", "hfx_create", "hfx_set_radial", "hfx_set_kpoint", "hfx_set_coulomb",
    "hfx_set_products", "hfx_get_products", "hfx_build_all", "hfx_build_exchange", "hfx_get_exchange",
    "hfx_exchange_device_ptr", "hfx_get_energy", "hfx_get_q0_bracket", "hfx_destroy", "hfx_strerror",
    "hfx_last_error", "hfx_version", "hfx_q0_bracket_noalloc", "hfx_get_transform",
    "hfx_set_overlap", "hfx_lapw_transform_all", "hfx_get_lapw_exchange", "hfx_set_momentum",
    "hfx_set_radial_functions", "hfx_get_radial_basis",
)


class HfxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class hfx_system(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_double * 9),
        ("n_atoms", ctypes.c_int),
        ("pos_frac", ctypes.c_void_p),
        ("rmt", ctypes.c_void_p),
        ("lmax", ctypes.c_int),
        ("Lmax", ctypes.c_int),
        ("n_rad", ctypes.c_int),
        ("mesh", ctypes.c_int * 3),
    ]


class hfx_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("sparse", ctypes.c_int),
        ("q0_term", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("herm_tol", ctypes.c_double),
        ("sparse_tol", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("work_bytes", ctypes.c_size_t),
        ("use_graph", ctypes.c_int),
        ("tile_nb_zhy", ctypes.c_int),
        ("tile_nb_zipw", ctypes.c_int),
        ("kp_term", ctypes.c_int),
        ("kp_deg_tol", ctypes.c_double),
        ("test_fail_wait", ctypes.c_int),
        ("inversion", ctypes.c_int),
    ]


class hfx_stats(ctypes.Structure):
    _fields_ = [
        ("ms_total", ctypes.c_double),
        ("ms_stage1", ctypes.c_double),
        ("ms_contract", ctypes.c_double),
        ("ms_finish", ctypes.c_double),
        ("useful_flops", ctypes.c_double),
        ("n_pairs", ctypes.c_int),
        ("n_batches", ctypes.c_int),
        ("sparse_used", ctypes.c_int),
        ("n_launches", ctypes.c_int),
        ("ms_zipw", ctypes.c_double),
        ("ms_apply", ctypes.c_double),
        ("ms_zhy", ctypes.c_double),
        ("flops_apply", ctypes.c_double),
        ("flops_zhy", ctypes.c_double),
        ("flops_zipw", ctypes.c_double),
        ("graph_replayed", ctypes.c_int),
        ("tile_nb_zhy", ctypes.c_int),
        ("tile_nb_zipw", ctypes.c_int),
        ("flops_apply_exec", ctypes.c_double),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libhfx.so; raise if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    L.hfx_default_options.restype = None
    L.hfx_default_options.argtypes = [P(hfx_options)]
    L.hfx_create.restype = ip
    L.hfx_create.argtypes = [P(hfx_system), P(hfx_options), P(vp)]
    L.hfx_set_radial.restype = ip
    L.hfx_set_radial.argtypes = [vp, ip, vp, vp]
    L.hfx_set_kpoint.restype = ip
    L.hfx_set_kpoint.argtypes = [vp, ip, ip, ip, ip, vp, vp, vp]
    L.hfx_set_coulomb.restype = ip
    L.hfx_set_coulomb.argtypes = [vp, ip, ip, vp, vp, ip, ip]
    L.hfx_get_transform.restype = ip
    L.hfx_get_transform.argtypes = [vp, ip, ip, vp]
    L.hfx_set_momentum.restype = ip
    L.hfx_set_momentum.argtypes = [vp, ip, vp, vp]
    L.hfx_set_overlap.restype = ip
    L.hfx_set_overlap.argtypes = [vp, ip, vp, ip]
    L.hfx_lapw_transform_all.restype = ip
    L.hfx_lapw_transform_all.argtypes = [vp, P(hfx_stats)]
    L.hfx_get_lapw_exchange.restype = ip
    L.hfx_get_lapw_exchange.argtypes = [vp, ip, vp, ip]
    L.hfx_set_products.restype = ip
    L.hfx_set_products.argtypes = [vp, ip, ip, vp]
    L.hfx_get_products.restype = ip
    L.hfx_get_products.argtypes = [vp, ip, ip, vp]
    L.hfx_build_all.restype = ip
    L.hfx_build_all.argtypes = [vp, ip, P(hfx_stats)]
    L.hfx_build_exchange.restype = ip
    L.hfx_build_exchange.argtypes = [vp, ip, vp, P(hfx_stats)]
    L.hfx_get_exchange.restype = ip
    L.hfx_get_exchange.argtypes = [vp, ip, vp]
    L.hfx_exchange_device_ptr.restype = ip
    L.hfx_exchange_device_ptr.argtypes = [vp, ip, P(vp)]
    L.hfx_get_energy.restype = ip
    L.hfx_get_energy.argtypes = [vp, P(dp)]
    L.hfx_get_q0_bracket.restype = ip
    L.hfx_get_q0_bracket.argtypes = [vp, P(dp)]
    L.hfx_destroy.restype = None
    L.hfx_destroy.argtypes = [vp]
    L.hfx_strerror.restype = ctypes.c_char_p
    L.hfx_strerror.argtypes = [ip]
    L.hfx_last_error.restype = ctypes.c_char_p
    L.hfx_last_error.argtypes = [vp]
    L.hfx_version.restype = ctypes.c_char_p
    L.hfx_version.argtypes = []
    L.hfx_set_radial_functions.restype = ip
    L.hfx_set_radial_functions.argtypes = [vp, ip, ip, vp, vp, vp, dp]
    L.hfx_get_radial_basis.restype = ip
    L.hfx_get_radial_basis.argtypes = [vp, ip, vp, vp, vp, vp]
    L.hfx_q0_bracket_noalloc.restype = ip
    L.hfx_q0_bracket_noalloc.argtypes = [vp, vp, dp, vp, vp]
    _lib = L
    return L


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _check(ctx, code: int):
    if code != HFX_OK:
        L = load()
        msg = L.hfx_last_error(ctx).decode() if ctx else ""
        raise HfxError(code, f"{L.hfx_strerror(code).decode()}: {msg}")


# ----------------------------------------------------------- same-name wrappers

def hfx_default_options() -> hfx_options:
    o = hfx_options()
    load().hfx_default_options(ctypes.byref(o))
    return o


def hfx_create(lattice, pos_frac, rmt, lmax, Lmax, n_rad, mesh, opt: Optional[hfx_options] = None):
    L = load()
    pos = _c(pos_frac, np.float64)
    rm = _c(rmt, np.float64)
    s = hfx_system()
    s.lattice[:] = [float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()]
    s.n_atoms = int(pos.shape[0])
    s.pos_frac = pos.ctypes.data
    s.rmt = rm.ctypes.data
    s.lmax, s.Lmax, s.n_rad = int(lmax), int(Lmax), int(n_rad)
    s.mesh[:] = [int(x) for x in mesh]
    if opt is None:
        opt = hfx_default_options()
    h = ctypes.c_void_p()
    code = L.hfx_create(ctypes.byref(s), ctypes.byref(opt), ctypes.byref(h))
    if code != HFX_OK:
        raise HfxError(code, L.hfx_strerror(code).decode())
    return h


def hfx_set_radial(ctx, atom: int, R, mu):
    R = _c(R, np.float64)
    mu = _c(mu, np.float64)
    _check(ctx, load().hfx_set_radial(ctx, int(atom), R.ctypes.data, mu.ctypes.data))


def hfx_set_radial_functions(ctx, atom: int, r, w, u, threshold: float = 1e-4):
    """u: (2(lmax+1), n_r) radial functions on the grid r with weights w."""
    r = _c(r, np.float64)
    w = _c(w, np.float64)
    u = _c(u, np.float64)
    _check(ctx, load().hfx_set_radial_functions(ctx, int(atom), int(r.size), r.ctypes.data, w.ctypes.data,
                                                u.ctypes.data, float(threshold)))


def hfx_get_radial_basis(ctx, atom: int, n_r: int, lmax: int, Lmax: int, P: int) -> dict:
    nlp = 2 * (lmax + 1)
    M = np.zeros(((Lmax + 1) * P, n_r))
    mu = np.zeros((Lmax + 1) * P)
    R = np.zeros(((Lmax + 1) * P, nlp, nlp))
    C = np.zeros((Lmax + 1, P, P))
    _check(ctx, load().hfx_get_radial_basis(ctx, int(atom), M.ctypes.data, mu.ctypes.data, R.ctypes.data,
                                            C.ctypes.data))
    return {"M": M, "mu": mu, "R": R, "C": C}


def hfx_set_kpoint(ctx, ik: int, n_bands: int, n_occ: int, G, c, A):
    G = _c(G, np.int32)
    c = _c(c, np.complex128)
    A = _c(A, np.complex128)
    _check(ctx, load().hfx_set_kpoint(ctx, int(ik), int(n_bands), int(n_occ), int(G.shape[0]), G.ctypes.data,
                                      c.ctypes.data, A.ctypes.data))


def hfx_set_coulomb(ctx, iq: int, G_aux, v, ld: Optional[int] = None, layout: int = HFX_LAYOUT_DENSE):
    """v: (N_aux, N_aux) complex, or a (N_aux, ld) array whose first N_aux
    columns hold the matrix (row stride ld)."""
    G = _c(G_aux, np.int32).reshape(-1, 3)
    v = _c(v, np.complex128)
    ld = int(v.shape[1]) if ld is None else int(ld)
    _check(ctx, load().hfx_set_coulomb(ctx, int(iq), int(G.shape[0]), G.ctypes.data if G.size else None,
                                       v.ctypes.data, ld, int(layout)))


def hfx_get_transform(ctx, atom: int, L: int, P: int) -> np.ndarray:
    out = np.zeros((P, P), np.float64)
    _check(ctx, load().hfx_get_transform(ctx, int(atom), int(L), out.ctypes.data))
    return out


def hfx_set_products(ctx, ik: int, iq: int, Z):
    if Z is None:
        _check(ctx, load().hfx_set_products(ctx, int(ik), int(iq), None))
        return
    Z = _c(Z, np.complex128)
    _check(ctx, load().hfx_set_products(ctx, int(ik), int(iq), Z.ctypes.data))


def hfx_get_products(ctx, ik: int, iq: int, shape) -> np.ndarray:
    out = np.zeros(shape, np.complex128)
    _check(ctx, load().hfx_get_products(ctx, int(ik), int(iq), out.ctypes.data))
    return out


def hfx_build_all(ctx, keep_products: bool = False) -> dict:
    st = hfx_stats()
    _check(ctx, load().hfx_build_all(ctx, int(bool(keep_products)), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in hfx_stats._fields_}


def hfx_build_exchange(ctx, ik: int, n_bands: int, stats: bool = False):
    """V^x(k) of one k (its N_k pairs); with stats=True also the build statistics."""
    out = np.zeros((n_bands, n_bands), np.complex128)
    st = hfx_stats()
    _check(ctx, load().hfx_build_exchange(ctx, int(ik), out.ctypes.data, ctypes.byref(st)))
    if stats:
        return out, {f: getattr(st, f) for f, _ in hfx_stats._fields_}
    return out


def hfx_get_exchange(ctx, ik: int, n_bands: int) -> np.ndarray:
    out = np.zeros((n_bands, n_bands), np.complex128)
    _check(ctx, load().hfx_get_exchange(ctx, int(ik), out.ctypes.data))
    return out


def hfx_exchange_device_ptr(ctx, ik: int) -> int:
    p = ctypes.c_void_p()
    _check(ctx, load().hfx_exchange_device_ptr(ctx, int(ik), ctypes.byref(p)))
    return int(p.value)


def hfx_get_energy(ctx) -> float:
    e = ctypes.c_double()
    _check(ctx, load().hfx_get_energy(ctx, ctypes.byref(e)))
    return float(e.value)


def hfx_get_q0_bracket(ctx) -> float:
    b = ctypes.c_double()
    _check(ctx, load().hfx_get_q0_bracket(ctx, ctypes.byref(b)))
    return float(b.value)


def hfx_q0_bracket_noalloc(lattice, mesh, beta: float, bracket_dev_ptr: int, stream: Optional[int] = None):
    """Allocation-free q->0 bracket: writes one double to the caller-owned
    device address ``bracket_dev_ptr`` (see include/hfx.h)."""
    lat = _c(lattice, np.float64).ravel()
    m = _c(mesh, np.int32).ravel()
    code = load().hfx_q0_bracket_noalloc(lat.ctypes.data, m.ctypes.data, float(beta), int(bracket_dev_ptr), stream)
    if code != HFX_OK:
        raise HfxError(code, load().hfx_strerror(code).decode())


def hfx_set_momentum(ctx, ik: int, eps, p):
    eps = _c(eps, np.float64)
    p = _c(p, np.complex128)
    _check(ctx, load().hfx_set_momentum(ctx, int(ik), eps.ctypes.data, p.ctypes.data))


def hfx_set_overlap(ctx, ik: int, S, ld: Optional[int] = None):
    S = _c(S, np.complex128)
    _check(ctx, load().hfx_set_overlap(ctx, int(ik), S.ctypes.data, int(S.shape[1]) if ld is None else int(ld)))


def hfx_lapw_transform_all(ctx) -> dict:
    st = hfx_stats()
    _check(ctx, load().hfx_lapw_transform_all(ctx, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in hfx_stats._fields_}


def hfx_get_lapw_exchange(ctx, ik: int, npw: int) -> np.ndarray:
    out = np.zeros((npw, npw), np.complex128)
    _check(ctx, load().hfx_get_lapw_exchange(ctx, int(ik), out.ctypes.data, int(npw)))
    return out


def hfx_destroy(ctx):
    if ctx:
        load().hfx_destroy(ctx)


def hfx_version() -> str:
    return load().hfx_version().decode()


# ----------------------------------------------------------- convenience class

class Context:
    """One exchange-matrix context bound to a system from ``synthetic``."""

    def __init__(self, sysm, precision: str = "sliced", sparse: str = "auto", q0_term: bool = True,
                 beta: float = 0.005, stream: Optional[int] = None, device: int = 0, work_bytes: int = 0,
                 use_graph: bool = True, tile_nb_zhy: int = 0, tile_nb_zipw: int = 0, test_fail_wait: bool = False,
                 tuning: bool = False, kp_term: bool = False, inversion: Optional[bool] = None):
        """tuning: take the tile shapes of this size class from the autotuner's
        file (paper_1003_0524_gb300/tuning.json) when it has them.
        inversion: the real-valued path of an inversion-symmetric system
        (default: what the system says, ``sysm.inversion``)."""
        self.tuned = None
        if tuning and not tile_nb_zhy and not tile_nb_zipw:
            from .autotune import lookup
            self.tuned = lookup(sysm)
            if self.tuned:
                tile_nb_zhy = int(self.tuned["tile_nb_zhy"])
                tile_nb_zipw = int(self.tuned["tile_nb_zipw"])
        opt = hfx_default_options()
        opt.precision = {"fp64": HFX_PREC_FP64, "sliced": HFX_PREC_SLICED}[precision]
        opt.sparse = {"auto": HFX_SPARSE_AUTO, "on": HFX_SPARSE_ON, "off": HFX_SPARSE_OFF}[sparse]
        opt.q0_term = int(bool(q0_term))
        opt.beta = float(beta)
        opt.stream = stream
        opt.device = int(device)
        opt.work_bytes = int(work_bytes)
        opt.use_graph = int(bool(use_graph))
        opt.tile_nb_zhy = int(tile_nb_zhy)
        opt.tile_nb_zipw = int(tile_nb_zipw)
        opt.test_fail_wait = int(bool(test_fail_wait))
        opt.kp_term = int(bool(kp_term))
        opt.inversion = int(bool(getattr(sysm, "inversion", False) if inversion is None else inversion))
        self.sys = sysm
        self.ctx = hfx_create(sysm.lattice, sysm.pos_frac, sysm.rmt, sysm.lmax, sysm.Lmax, sysm.P, sysm.mesh, opt)

    def load_system(self, kpoints: bool = True, coulomb: bool = True, radial: bool = True):
        s = self.sys
        if radial:
            for a in range(s.n_atoms):
                hfx_set_radial(self.ctx, a, s.R[a], s.mu[a])
        if kpoints:
            self.set_kpoints()
        if coulomb:
            for iq in range(s.n_k):
                hfx_set_coulomb(self.ctx, iq, s.Gaux[iq], s.v[iq])

    def set_kpoints(self):
        s = self.sys
        for ik in range(s.n_k):
            hfx_set_kpoint(self.ctx, ik, int(s.n_bands[ik]), int(s.n_occ[ik]), s.Gk[ik], s.c[ik], s.A[ik])

    def build_all(self, keep_products: bool = False) -> dict:
        return hfx_build_all(self.ctx, keep_products)

    def exchange(self, ik: int) -> np.ndarray:
        return hfx_get_exchange(self.ctx, ik, int(self.sys.n_bands[ik]))

    def build_exchange(self, ik: int, stats: bool = False):
        return hfx_build_exchange(self.ctx, ik, int(self.sys.n_bands[ik]), stats)

    def energy(self) -> float:
        return hfx_get_energy(self.ctx)

    def q0_bracket(self) -> float:
        return hfx_get_q0_bracket(self.ctx)

    def products(self, ik: int, iq: int, ikp: int) -> np.ndarray:
        s = self.sys
        return hfx_get_products(self.ctx, ik, iq, (s.n_aux(iq), int(s.n_occ[ikp]), int(s.n_bands[ik])))

    def set_products(self, ik: int, iq: int, Z):
        hfx_set_products(self.ctx, ik, iq, Z)

    def close(self):
        if self.ctx:
            hfx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
