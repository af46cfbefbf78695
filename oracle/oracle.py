"""Python binding of the FP64 CPU oracle (oracle/hfx_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports, links or runs anything in this directory.

The binding only marshals numpy arrays into the C struct; every number is
computed by the C code, except one change of basis: for inversion-symmetric
inputs (Sec. III.D) the Coulomb matrices arrive in the symmetrized MT basis
and are taken back to the original one as v = S v' S^H with the matrix S of
``ora_sym_matrix`` (a plain matrix product).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhfx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OraSys(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_double * 9),
        ("n_atoms", ctypes.c_int),
        ("pos_frac", ctypes.c_void_p),
        ("rmt", ctypes.c_void_p),
        ("lmax", ctypes.c_int),
        ("Lmax", ctypes.c_int),
        ("P", ctypes.c_int),
        ("mesh", ctypes.c_int * 3),
        ("n_bands", ctypes.c_void_p),
        ("n_occ", ctypes.c_void_p),
        ("npw", ctypes.c_void_p),
        ("pw_off", ctypes.c_void_p),
        ("Gk", ctypes.c_void_p),
        ("c_off", ctypes.c_void_p),
        ("c", ctypes.c_void_p),
        ("A_off", ctypes.c_void_p),
        ("A", ctypes.c_void_p),
        ("R", ctypes.c_void_p),
        ("mu", ctypes.c_void_p),
        ("n_ipw", ctypes.c_void_p),
        ("gaux_off", ctypes.c_void_p),
        ("Gaux", ctypes.c_void_p),
        ("v_off", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("beta", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            L.ora_gaunt.restype = dp
            L.ora_gaunt.argtypes = [ip] * 6
            L.ora_threej.restype = dp
            L.ora_threej.argtypes = [ip] * 6
            L.ora_omega.restype = dp
            L.ora_omega.argtypes = [vp]
            L.ora_theta.restype = None
            L.ora_theta.argtypes = [vp, ip, vp, vp]
            L.ora_fold.restype = None
            L.ora_fold.argtypes = [vp, ip, ip, vp, vp]
            for name in ("ora_zmt", "ora_zipw", "ora_zipw_direct"):
                f = getattr(L, name)
                f.restype = ip
                f.argtypes = [vp, ip, ip, vp]
            L.ora_transform_T.restype = None
            L.ora_transform_T.argtypes = [ip, vp, vp]
            L.ora_vdiv.restype = dp
            L.ora_vdiv.argtypes = [vp]
            L.ora_vx.restype = ip
            L.ora_vx.argtypes = [vp, ip, ip, ip, vp]
            L.ora_vx_sub.restype = ip
            L.ora_vx_sub.argtypes = [vp, ip, ip, vp, ip, vp]
            L.ora_vx_part.restype = ip
            L.ora_vx_part.argtypes = [vp, ip, ip, vp, ip, vp, vp]
            L.ora_lapw_trafo.restype = ip
            L.ora_lapw_trafo.argtypes = [ip, ip, vp, vp, vp, vp]
            L.ora_kp_term.restype = ip
            L.ora_kp_term.argtypes = [ip, ip, vp, vp, dp, dp, vp]
            L.ora_inv_partner.restype = ip
            L.ora_inv_partner.argtypes = [vp, vp]
            L.ora_sym_matrix.restype = ip
            L.ora_sym_matrix.argtypes = [vp, ip, vp]
            L.ora_radial_coulomb.restype = dp
            L.ora_radial_coulomb.argtypes = [ip, vp, vp, ip, vp, vp]
            L.ora_mpb_radial.restype = ip
            L.ora_mpb_radial.argtypes = [ip, vp, vp, vp, ip, ip, ip, dp, vp, vp, vp, vp]
            L.ora_num_threads.restype = ip
            L.ora_num_threads.argtypes = []
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Oracle:
    """Holds contiguous copies of a System's arrays and the C struct."""

    def __init__(self, sysm, beta: float = 0.005):
        self.sys = sysm
        L = lib()
        self._L = L
        nk = sysm.n_k
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a

        self.n_bands = arr(sysm.n_bands, np.int32)
        self.n_occ = arr(sysm.n_occ, np.int32)
        self.npw = arr([g.shape[0] for g in sysm.Gk], np.int32)
        self.pw_off = arr(np.concatenate([[0], np.cumsum(self.npw)[:-1]]), np.int64)
        self.Gk = arr(np.concatenate(sysm.Gk, axis=0), np.int32)
        csz = [c.size for c in sysm.c]
        self.c_off = arr(np.concatenate([[0], np.cumsum(csz)[:-1]]), np.int64)
        self.c = arr(np.concatenate([c.ravel() for c in sysm.c]), np.complex128)
        asz = [a.size for a in sysm.A]
        self.A_off = arr(np.concatenate([[0], np.cumsum(asz)[:-1]]), np.int64)
        self.A = arr(np.concatenate([a.ravel() for a in sysm.A]), np.complex128)
        self.R = arr(sysm.R, np.float64)
        self.mu = arr(sysm.mu, np.float64)
        self.n_ipw = arr([g.shape[0] for g in sysm.Gaux], np.int32)
        self.gaux_off = arr(np.concatenate([[0], np.cumsum(self.n_ipw)[:-1]]), np.int64)
        self.Gaux = arr(np.concatenate(sysm.Gaux, axis=0) if sum(self.n_ipw) else
                        np.zeros((1, 3)), np.int32)
        vsz = [v.size for v in sysm.v]
        self.v_off = arr(np.concatenate([[0], np.cumsum(vsz)[:-1]]), np.int64)
        self.v = arr(np.concatenate([v.ravel() for v in sysm.v]), np.complex128)
        self.pos = arr(sysm.pos_frac, np.float64)
        self.rmt = arr(sysm.rmt, np.float64)
        self._keep = keep
        s = OraSys()
        s.lattice[:] = list(np.asarray(sysm.lattice, dtype=np.float64).ravel())
        s.n_atoms = sysm.n_atoms
        s.pos_frac = _ptr(self.pos)
        s.rmt = _ptr(self.rmt)
        s.lmax, s.Lmax, s.P = sysm.lmax, sysm.Lmax, sysm.P
        s.mesh[:] = list(sysm.mesh)
        for name in ("n_bands", "n_occ", "npw", "pw_off", "Gk", "c_off", "c", "A_off", "A", "R",
                     "mu", "n_ipw", "gaux_off", "Gaux", "v_off", "v"):
            setattr(s, name, _ptr(getattr(self, name)))
        s.beta = beta
        self.s = s
        self._sp = ctypes.byref(s)
        assert nk == len(sysm.Gk)
        if getattr(sysm, "inversion", False):
            # v(q) is given over the symmetrized MT functions: v = S v' S^H
            S = self.sym_matrix()
            nmt = sysm.n_mt
            full = []
            for vq in sysm.v:
                w = np.array(vq, dtype=np.complex128)
                w[:nmt, :] = S @ w[:nmt, :]
                w[:, :nmt] = w[:, :nmt] @ S.conj().T
                full.append(w)
            self.v = arr(np.concatenate([w.ravel() for w in full]), np.complex128)
            s.v = _ptr(self.v)

    def inv_partner(self) -> np.ndarray:
        """Partner atom of every atom under r -> -r (-1 where none)."""
        out = np.zeros(self.sys.n_atoms, np.int32)
        self._L.ora_inv_partner(self._sp, _ptr(out))
        return out

    def sym_matrix(self, n_aux: int | None = None) -> np.ndarray:
        """S with M'_J = sum_I S[I, J] M_I (Eqs. sym MT functions) over the
        first n_aux functions of the MPB (default: the MT functions)."""
        n = self.sys.n_mt if n_aux is None else int(n_aux)
        S = np.zeros((n, n), np.complex128)
        if self._L.ora_sym_matrix(self._sp, n, _ptr(S)) != 0:
            raise ValueError("an atom has no inversion partner")
        return S

    # -- thin wrappers ---------------------------------------------------
    def omega(self) -> float:
        return self._L.ora_omega(self._sp)

    def fold(self, ik: int, iq: int):
        ikp = np.zeros(1, np.int32)
        G0 = np.zeros(3, np.int32)
        self._L.ora_fold(self._sp, ik, iq, _ptr(ikp), _ptr(G0))
        return int(ikp[0]), G0.copy()

    def theta(self, K) -> np.ndarray:
        K = np.ascontiguousarray(np.asarray(K, dtype=np.int32).reshape(-1, 3))
        out = np.zeros(K.shape[0], np.complex128)
        self._L.ora_theta(self._sp, K.shape[0], _ptr(K), _ptr(out))
        return out

    def _zshape(self, ik, iq, rows):
        ikp, _ = self.fold(ik, iq)
        return (rows, int(self.sys.n_occ[ikp]), int(self.sys.n_bands[ik]))

    def zmt(self, ik: int, iq: int) -> np.ndarray:
        out = np.zeros(self._zshape(ik, iq, self.sys.n_mt), np.complex128)
        self._L.ora_zmt(self._sp, ik, iq, _ptr(out))
        return out

    def zipw(self, ik: int, iq: int, direct: bool = False) -> np.ndarray:
        out = np.zeros(self._zshape(ik, iq, int(self.n_ipw[iq])), np.complex128)
        f = self._L.ora_zipw_direct if direct else self._L.ora_zipw
        f(self._sp, ik, iq, _ptr(out))
        return out

    def z(self, ik: int, iq: int) -> np.ndarray:
        return np.concatenate([self.zmt(ik, iq), self.zipw(ik, iq)], axis=0)

    def vdiv(self) -> float:
        return self._L.ora_vdiv(self._sp)

    def vx(self, ik: int, transformed: bool = False, q0term: bool = True) -> np.ndarray:
        nb = int(self.sys.n_bands[ik])
        out = np.zeros((nb, nb), np.complex128)
        self._L.ora_vx(self._sp, ik, int(transformed), int(q0term), _ptr(out))
        return out


    def vx_sub(self, ik: int, bands, q0term: bool = True) -> np.ndarray:
        """The sub-block V^x(k)[bands][bands] (every occupied band of k - q
        in the m sum), at the cost of len(bands) bands."""
        sel = np.ascontiguousarray(np.asarray(bands, dtype=np.int32).ravel())
        out = np.zeros((sel.size, sel.size), np.complex128)
        rc = self._L.ora_vx_sub(self._sp, ik, int(sel.size), _ptr(sel), int(q0term), _ptr(out))
        if rc != 0:
            raise ValueError("band index out of range")
        return out


    def vx_part(self, ik: int, bands, qs) -> np.ndarray:
        """The terms of the q in qs of the sub-block vx_sub(ik, bands), without
        the q->0 term (a bounded piece of the q sum, for timing)."""
        sel = np.ascontiguousarray(np.asarray(bands, dtype=np.int32).ravel())
        ql = np.ascontiguousarray(np.asarray(qs, dtype=np.int32).ravel())
        out = np.zeros((sel.size, sel.size), np.complex128)
        rc = self._L.ora_vx_part(self._sp, ik, int(sel.size), _ptr(sel), int(ql.size), _ptr(ql), _ptr(out))
        if rc != 0:
            raise ValueError("band or q index out of range")
        return out


def gaunt(L, M, l1, m1, l2, m2) -> float:
    return lib().ora_gaunt(L, M, l1, m1, l2, m2)


def threej(j1, j2, j3, m1, m2, m3) -> float:
    return lib().ora_threej(j1, j2, j3, m1, m2, m3)


def transform_T(mu) -> np.ndarray:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    P = mu.shape[0]
    T = np.zeros((P, P), np.float64)
    lib().ora_transform_T(P, _ptr(mu), _ptr(T))
    return T


def lapw_trafo(S, c, V) -> np.ndarray:
    """Eq. (APW trafo): V_GG' = (S c) V (c^H S) with S (npw x npw), c (nb x npw)
    the coefficients of the bands in the basis of k, V (nb x nb)."""
    S = np.ascontiguousarray(S, dtype=np.complex128)
    c = np.ascontiguousarray(c, dtype=np.complex128)
    V = np.ascontiguousarray(V, dtype=np.complex128)
    nb, npw = c.shape
    assert S.shape == (npw, npw) and V.shape == (nb, nb)
    out = np.zeros((npw, npw), np.complex128)
    lib().ora_lapw_trafo(npw, nb, _ptr(S), _ptr(c), _ptr(V), _ptr(out))
    return out


def kp_term(eps, p, nocc: int, nk_omega: float, deg_tol: float = 1e-6) -> np.ndarray:
    """Appendix A: the k.p term at q = 0 added to V^x(k), -Abar / (N_k Omega),
    from the band energies eps (nb) and momentum elements p (3, nb, nb)."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.complex128)
    nb = eps.size
    assert p.shape == (3, nb, nb)
    out = np.zeros((nb, nb), np.complex128)
    lib().ora_kp_term(nb, int(nocc), _ptr(eps), _ptr(p), float(nk_omega), float(deg_tol), _ptr(out))
    return out


def radial_coulomb(r, w, L: int, f, g) -> float:
    """4 pi/(2L+1) int int f(r) g(r') r<^L/r>^(L+1) r^2 r'^2 dr dr' on the grid."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    return lib().ora_radial_coulomb(r.size, _ptr(r), _ptr(w), int(L), _ptr(f), _ptr(g))


def mpb_radial(r, w, u, lmax: int, Lmax: int, P: int, thr: float = 1e-4) -> dict:
    """Sec. III.B: the MT product basis of one atom from its radial functions
    u [2(lmax+1)][n_r] on the grid r with weights w: M [(Lmax+1) P][n_r], the
    multipole moments mu, the radial integrals R and the on-site Coulomb blocks
    C [(Lmax+1)][P][P].  Raises if fewer than P functions survive for some L."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = r.size
    nlp = 2 * (lmax + 1)
    assert u.shape == (nlp, n)
    M = np.zeros(((Lmax + 1) * P, n))
    mu = np.zeros((Lmax + 1) * P)
    R = np.zeros(((Lmax + 1) * P, nlp, nlp))
    C = np.zeros((Lmax + 1, P, P))
    rc = lib().ora_mpb_radial(n, _ptr(r), _ptr(w), _ptr(u), lmax, Lmax, P, float(thr), _ptr(M), _ptr(mu), _ptr(R),
                              _ptr(C))
    if rc != 0:
        raise ValueError(f"fewer than P product functions above the threshold for L = {-rc - 1}")
    return {"M": M, "mu": mu, "R": R, "C": C}


def num_threads() -> int:
    return lib().ora_num_threads()


def exchange_energy(sysm, V) -> float:
    """E_x per spin channel from the diagonal of V^x:
    (1/2)(1/N_k) sum_k sum_n f_nk Re V_nn(k), f_nk = 1 for n < n_occ(k)."""
    tot = 0.0
    for ik, Vk in V.items():
        no = int(sysm.n_occ[ik])
        tot += float(np.real(np.trace(Vk[:no, :no])))
    return 0.5 * tot / sysm.n_k
