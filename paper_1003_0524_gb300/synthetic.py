"""Seeded synthetic inputs for the nonlocal exchange-matrix build.

This module produces DATA ONLY: crystal geometry, plane-wave lists, random
wave-function coefficients, random radial product integrals and multipole
moments, and random Hermitian positive-definite Coulomb matrices with the
block structure that the multipole transformation of Sec. III.C (Fig. 1)
produces.  It contains none of the exchange-matrix arithmetic: no Gaunt
coefficients, no step function, no projections, no vector-matrix-vector
products, no q->0 term.  Both the FP64 CPU oracle (``oracle/``) and the CUDA
library consume what it returns.

Conventions (shared by every consumer):

* lattice rows a_i in bohr, reciprocal rows b_i with a_i . b_j = 2 pi delta_ij;
* Gamma-centred k mesh, k = sum_i (j_i / N_i) b_i, flat index
  ik = (j_0 * N_1 + j_1) * N_2 + j_2; the q mesh is the same set (Sec. III.C
  requires k - q to be a mesh point again);
* LAPW MT index lmp = 2 * (l*l + l + m) + p, p in {0, 1} (u and u-dot,
  Eq. FLAPW-basis), N_lmp = 2 (lmax+1)^2;
* radial index lp = 2*l + p;
* MT product-basis index inside one atom LMP = (L*L + L + M) * P + P_index;
  atoms are outermost, then the interstitial plane waves follow in the order
  of the per-q list (Sec. III.B);
* complex arrays are numpy complex128, row-major;
* per-k arrays: c[k] shape (n_bands, npw), A[k] shape (n_bands, n_atoms, N_lmp);
* R shape (n_atoms, (Lmax+1)*P, 2(lmax+1), 2(lmax+1)), symmetric in its last
  two indices; mu shape (n_atoms, (Lmax+1)*P);
* v[q] shape (N_aux(q), N_aux(q)), Hermitian positive definite, in the
  original (untransformed) basis ordering above.

Inversion-symmetric variants (``make_system(cfg, inversion=True)``, Sec. III.D):
the atoms come in pairs a, a' with R_a' = -R_a up to a lattice vector T_a
(an atom at an inversion centre is its own partner), partners share sphere
radius, radial integrals and multipole moments, and the wave functions obey
phi(-r) = phi(r)^*: real plane-wave coefficients and, with
psi(R_a + T + x) = e^{ik.T} sum_lmp A^a_lmp u_lp(|x|) Y_lm(x) inside the spheres,
A^{a'}_{l,-m,p} = (-1)^(l+m) e^{ik.T_a} conj(A^a_{lmp}).  v[q] is then given
over the symmetrized MT functions of Eqs. (sym MT functions) (same labels,
pairs ordered with the lower atom index first, M < 0 first on an atom at an
inversion centre): a real symmetric positive-definite matrix with the block
structure of Fig. 1, partner channels sharing their on-site blocks.

Workload recipes follow the paper's systems in shape only (Sec. IV: cell sizes,
2-10 atoms, Lmax = 4..5, band windows of tens to hundreds of bands, k meshes
up to 6x6x6).  The paper's own crystals and FLEUR wave functions are not
available; every value here is drawn from a seeded PCG64 stream.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 1003052400
ANGSTROM = 1.0 / 0.529177210903  # bohr per angstrom


def _cubic(a: float) -> np.ndarray:
    return np.eye(3) * a


def _rhombohedral(a: float, alpha_deg: float) -> np.ndarray:
    """Three equal axes of length a with pairwise angle alpha (rows)."""
    al = math.radians(alpha_deg)
    ca = math.cos(al)
    a1 = np.array([1.0, 0.0, 0.0])
    a2 = np.array([ca, math.sin(al), 0.0])
    cx = ca
    cy = (ca - ca * ca) / math.sin(al)
    cz = math.sqrt(max(0.0, 1.0 - cx * cx - cy * cy))
    a3 = np.array([cx, cy, cz])
    return a * np.stack([a1, a2, a3])


def _corundum_like_positions() -> List[List[float]]:
    u, x = 0.352, 0.556
    pos = []
    for s in (1.0, -1.0):
        pos.append([s * u, s * u, s * u])
        pos.append([s * (0.5 + u) % 1.0, s * (0.5 + u) % 1.0, s * (0.5 + u) % 1.0])
    for s in (1.0, -1.0):
        for perm in ((x, 0.5 - x, 0.25), (0.25, x, 0.5 - x), (0.5 - x, 0.25, x)):
            pos.append([(s * c) % 1.0 for c in perm])
    return pos


# Workload table.  "aux" is ("cut", G'max) for |q+G| <= G'max, or
# ("count", lo, hi) for a per-q count drawn from U{lo..hi} keeping the
# smallest |q+G|.  "a_scale" multiplies the MT coefficients A so that the
# muffin-tin and interstitial projections have comparable magnitude, and
# "scale" multiplies every Coulomb matrix so that the largest |V^x_nn| of the
# workload is of order 1 Ha (both fixed once from oracle runs).
CONFIGS = {
    0: dict(name="cubic_1atom_k2x2x2_n8", lattice=_cubic(8.0), pos=[[0.0, 0.0, 0.0]],
            rmt=[2.2], mesh=(2, 2, 2), nb=8, no=4, lmax=4, Lmax=4, P=2, gmax=3.0,
            aux=("cut", 2.5), sparse=False, a_scale=0.095, scale=19.7),
    1: dict(name="zincblende_2atom_k4x4x4_n40", lattice=_cubic(10.3),
            pos=[[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]], pos_inv=[[0.125, 0.125, 0.125], [-0.125, -0.125, -0.125]],
            rmt=[2.2, 2.2], mesh=(4, 4, 4),
            nb=40, no=8, lmax=4, Lmax=4, P=3, gmax=3.0, aux=("cut", 3.0), sparse=True,
            a_scale=0.065, scale=24.0),
    2: dict(name="zincblende_2atom_k4x4x4_uneven", lattice=_cubic(10.3),
            pos=[[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]], pos_inv=[[0.125, 0.125, 0.125], [-0.125, -0.125, -0.125]],
            rmt=[2.2, 2.2], mesh=(4, 4, 4),
            nb=("U", 32, 48), no=("U", 6, 10), lmax=4, Lmax=4, P=3, gmax=3.0,
            aux=("count", 520, 680), sparse=True, a_scale=0.065, scale=24.0),
    3: dict(name="perovskite_5atom_k6x6x6_n120", lattice=_cubic(7.4),
            pos=[[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5],
                 [0.0, 0.5, 0.5]],
            rmt=[2.4, 1.8, 1.5, 1.5, 1.5], mesh=(6, 6, 6), nb=120, no=20, lmax=4,
            Lmax=4, P=3, gmax=3.0, aux=("count", 1100, 1100), sparse=True, a_scale=0.17,
            scale=0.223),
    4: dict(name="corundum_10atom_k4x4x4_n250",
            lattice=_rhombohedral(5.3 * ANGSTROM, 55.3), pos=_corundum_like_positions(),
            rmt=[1.7] * 4 + [1.35] * 6, mesh=(4, 4, 4), nb=250, no=48, lmax=4, Lmax=5,
            P=2, gmax=3.0, aux=("count", 2300, 2300), sparse=True, a_scale=0.15, scale=0.122),
}


@dataclasses.dataclass
class System:
    """All inputs of one exchange-matrix build (one spin channel)."""
    name: str
    lattice: np.ndarray          # (3,3) rows a_i, bohr
    pos_frac: np.ndarray         # (n_atoms, 3)
    rmt: np.ndarray              # (n_atoms,)
    lmax: int
    Lmax: int
    P: int
    mesh: tuple
    gmax: float
    n_bands: np.ndarray          # (N_k,) int
    n_occ: np.ndarray            # (N_k,) int
    Gk: List[np.ndarray]         # per k: (npw, 3) int32
    c: List[np.ndarray]          # per k: (n_bands, npw) complex128
    A: List[np.ndarray]          # per k: (n_bands, n_atoms, N_lmp) complex128
    R: np.ndarray                # (n_atoms, (Lmax+1)P, 2(lmax+1), 2(lmax+1))
    mu: np.ndarray               # (n_atoms, (Lmax+1)P)
    Gaux: List[np.ndarray]       # per q: (n_ipw, 3) int32
    v: List[np.ndarray]          # per q: (N_aux, N_aux) complex128
    sparse: bool
    scale: float
    seed: int
    inversion: bool = False      # v over the symmetrized MT functions (Sec. III.D)

    @property
    def n_atoms(self) -> int:
        return int(self.pos_frac.shape[0])

    @property
    def n_k(self) -> int:
        return int(np.prod(self.mesh))

    @property
    def n_lmp(self) -> int:
        return 2 * (self.lmax + 1) ** 2

    @property
    def n_mt(self) -> int:
        return self.n_atoms * (self.Lmax + 1) ** 2 * self.P

    def n_aux(self, iq: int) -> int:
        return self.n_mt + int(self.Gaux[iq].shape[0])

    def recip(self) -> np.ndarray:
        return reciprocal(self.lattice)

    def kpoint_frac(self, ik: int) -> np.ndarray:
        return kpoint_frac(self.mesh, ik)


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * math.pi * np.linalg.inv(lattice).T


def kpoint_index(mesh, j) -> int:
    return (int(j[0]) * mesh[1] + int(j[1])) * mesh[2] + int(j[2])


def kpoint_frac(mesh, ik: int) -> np.ndarray:
    j2 = ik % mesh[2]
    j1 = (ik // mesh[2]) % mesh[1]
    j0 = ik // (mesh[1] * mesh[2])
    return np.array([j0 / mesh[0], j1 / mesh[1], j2 / mesh[2]])


def _g_sphere(kfrac: np.ndarray, lattice: np.ndarray, radius: float) -> np.ndarray:
    B = reciprocal(lattice)
    bound = [int(math.ceil(radius * np.linalg.norm(lattice[i]) / (2 * math.pi))) + 2
             for i in range(3)]
    r = [np.arange(-b, b + 1) for b in bound]
    g = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    kc = (kfrac[None, :] + g) @ B
    nrm = np.sqrt((kc * kc).sum(axis=1))
    keep = nrm <= radius + 1e-12
    g, nrm = g[keep], nrm[keep]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], np.round(nrm, 12)))
    return g[order].astype(np.int32), nrm[order]


def _g_count(kfrac: np.ndarray, lattice: np.ndarray, count: int) -> np.ndarray:
    B = reciprocal(lattice)
    vol_g = abs(np.linalg.det(B))
    radius = (count * vol_g * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0) * 1.3 + 1.0
    g, nrm = _g_sphere(kfrac, lattice, radius)
    assert g.shape[0] >= count
    return g[:count].copy(), nrm[:count].copy()


def _cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex normal CN(0,1): real and imaginary parts N(0, 1/2)."""
    x = rng.standard_normal(shape)
    y = rng.standard_normal(shape)
    return (x + 1j * y) / math.sqrt(2.0)


def _haar_unitary(rng: np.random.Generator, n: int) -> np.ndarray:
    z = _cn(rng, (n, n))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def _haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * np.sign(d)[None, :]


def inversion_partners(pos_frac, rmt) -> np.ndarray:
    """Partner of every atom under r -> -r (fractional positions summing to
    integers, equal sphere radii); raises if an atom has none."""
    pos = np.asarray(pos_frac, dtype=np.float64)
    out = np.full(pos.shape[0], -1, dtype=np.int64)
    for a in range(pos.shape[0]):
        for b in range(pos.shape[0]):
            d = pos[a] + pos[b]
            if np.all(np.abs(d - np.round(d)) < 1e-8) and abs(rmt[a] - rmt[b]) < 1e-12:
                out[a] = b
                break
        if out[a] < 0:
            raise ValueError(f"atom {a} has no inversion partner")
    return out


def _frame_with_first_row(rng: np.random.Generator, mu: np.ndarray) -> np.ndarray:
    """A random real orthogonal P x P matrix whose first row is mu/|mu|.

    Built from a library QR of [mu, gaussian columns]; any orthonormal
    completion serves the generator (the consumers construct their own)."""
    P = mu.shape[0]
    m = np.concatenate([mu[:, None], rng.standard_normal((P, P - 1))], axis=1)
    q, _ = np.linalg.qr(m)
    if np.dot(q[:, 0], mu) < 0:
        q[:, 0] = -q[:, 0]
    return q.T.copy()


def overlap(sysm, ik: int, seed: Optional[int] = None) -> np.ndarray:
    """A seeded Hermitian positive-definite overlap matrix S_GG'(k) of the
    basis functions of k (npw x npw, in the order of sysm.Gk[ik]): the unit
    matrix plus a random positive semi-definite part of norm ~0.1, standing in
    for the LAPW overlap (interstitial step-function plus muffin-tin terms)."""
    npw = int(sysm.Gk[ik].shape[0])
    rng = np.random.Generator(np.random.PCG64((sysm.seed if seed is None else seed) * 1000 + 7 + ik))
    w = _cn(rng, (npw, npw))
    s = np.eye(npw) + 0.1 * (w @ w.conj().T) / npw
    return 0.5 * (s + s.conj().T)


def momentum(sysm, ik: int, seed: Optional[int] = None):
    """Seeded band energies (ascending, occupied below a gap of 0.2 Ha) and
    anti-Hermitian momentum matrix elements p[a][m][n] = <phi_m|d_a|phi_n>
    (a = x, y, z; entries ~0.3 bohr^-1) of the bands of k, standing in for the
    inputs of the k.p term at q = 0."""
    nb, no = int(sysm.n_bands[ik]), int(sysm.n_occ[ik])
    rng = np.random.Generator(np.random.PCG64((sysm.seed if seed is None else seed) * 1000 + 500 + ik))
    occ = np.sort(rng.uniform(-1.0, 0.0, no))
    emp = np.sort(rng.uniform(0.2, 2.0, nb - no))
    eps = np.concatenate([occ, emp])
    w = 0.3 * _cn(rng, (3, nb, nb))
    p = 0.5 * (w - np.conj(np.swapaxes(w, 1, 2)))
    return eps, p


def sphere_gap(lattice, pos_frac, rmt) -> float:
    """Smallest |R_i - R_j - T| - S_i - S_j over atom pairs and lattice shifts
    (negative means overlapping muffin-tin spheres)."""
    n = len(pos_frac)
    best = np.inf
    shifts = np.stack(np.meshgrid(*[np.arange(-2, 3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for i in range(n):
        for j in range(n):
            d = (np.asarray(pos_frac[j]) - np.asarray(pos_frac[i]))[None, :] + shifts
            dc = np.linalg.norm(d @ lattice, axis=1)
            if i == j:
                dc = dc[dc > 1e-9]
            best = min(best, float(dc.min()) - rmt[i] - rmt[j])
    return best


def make_system(cfg: int | dict, *, seed: Optional[int] = None, mesh=None, nb=None,
                no=None, aux=None, scale=None, inversion: bool = False) -> System:
    """Build the seeded synthetic inputs of a workload.

    ``cfg`` is an index into CONFIGS or a dict with the same keys.  Keyword
    overrides shrink a workload for tests (mesh, band counts, aux recipe).
    ``inversion`` draws the inversion-symmetric variant (module docstring):
    the positions of ``pos_inv`` where the workload gives one, its own seed."""
    if inversion:
        return _make_system_inv(cfg, seed=seed, mesh=mesh, nb=nb, no=no, aux=aux, scale=scale)
    if isinstance(cfg, int):
        index = cfg
        spec = dict(CONFIGS[cfg])
    else:
        index = 99
        spec = dict(cfg)
    for key, val in (("mesh", mesh), ("nb", nb), ("no", no), ("aux", aux), ("scale", scale)):
        if val is not None:
            spec[key] = val
    if seed is None:
        seed = SEED_BASE + index
    rng = np.random.Generator(np.random.PCG64(seed))

    lattice = np.asarray(spec["lattice"], dtype=np.float64)
    pos = np.asarray(spec["pos"], dtype=np.float64)
    rmt = np.asarray(spec["rmt"], dtype=np.float64)
    mesh_t = tuple(int(x) for x in spec["mesh"])
    n_k = int(np.prod(mesh_t))
    n_at = pos.shape[0]
    lmax, Lmax, P = int(spec["lmax"]), int(spec["Lmax"]), int(spec["P"])
    n_lmp = 2 * (lmax + 1) ** 2
    n_lp = 2 * (lmax + 1)
    nlm_aux = (Lmax + 1) ** 2

    if sphere_gap(lattice, pos, rmt) <= 0.0:
        raise ValueError("muffin-tin spheres overlap")
    # band windows
    def draw(spec_val):
        if isinstance(spec_val, tuple):
            return rng.integers(spec_val[1], spec_val[2] + 1, size=n_k)
        return np.full(n_k, int(spec_val))
    n_bands = draw(spec["nb"]).astype(np.int32)
    n_occ = draw(spec["no"]).astype(np.int32)
    n_occ = np.minimum(n_occ, n_bands)

    Gk, c, A = [], [], []
    for ik in range(n_k):
        kf = kpoint_frac(mesh_t, ik)
        g, _ = _g_sphere(kf, lattice, float(spec["gmax"]))
        Gk.append(g)
        npw = g.shape[0]
        c.append(_cn(rng, (int(n_bands[ik]), npw)) / math.sqrt(npw))
        A.append(_cn(rng, (int(n_bands[ik]), n_at, n_lmp)) * float(spec.get("a_scale", 1.0)))

    R = rng.standard_normal((n_at, (Lmax + 1) * P, n_lp, n_lp)) * 0.1
    R = np.triu(R) + np.swapaxes(np.triu(R, 1), -1, -2)
    mu = rng.standard_normal((n_at, (Lmax + 1) * P))

    aux_spec = spec["aux"]
    Gaux, gnorm = [], []
    if aux_spec[0] == "count":
        counts = rng.integers(aux_spec[1], aux_spec[2] + 1, size=n_k)
    for iq in range(n_k):
        qf = kpoint_frac(mesh_t, iq)
        if aux_spec[0] == "cut":
            g, nrm = _g_sphere(qf, lattice, float(aux_spec[1]))
        else:
            g, nrm = _g_count(qf, lattice, int(counts[iq]))
        Gaux.append(g)
        gnorm.append(nrm)
    gp_max = max(float(x.max()) if x.size else 0.0 for x in gnorm)

    s = float(spec["scale"])
    sparse = bool(spec["sparse"])
    frames = [[_frame_with_first_row(rng, mu[a, L * P:(L + 1) * P]) for L in range(Lmax + 1)]
              for a in range(n_at)] if sparse else None
    v = []
    n_mt = n_at * nlm_aux * P
    for iq in range(n_k):
        n_ipw = Gaux[iq].shape[0]
        if not sparse:
            n = n_mt + n_ipw
            kappa = rng.uniform(0.0, gp_max, size=n_mt)
            g = np.concatenate([kappa, gnorm[iq]])
            d = s * 4.0 * math.pi / (g * g + 0.05)
            U = _haar_unitary(rng, n)
            vq = (U * d[None, :]) @ U.conj().T
            v.append(0.5 * (vq + vq.conj().T))
            continue
        D = n_at * nlm_aux + n_ipw
        kappa = rng.uniform(0.0, gp_max, size=n_at * nlm_aux)
        g = np.concatenate([kappa, gnorm[iq]])
        d = s * 4.0 * math.pi / (g * g + 0.05)
        U = _haar_unitary(rng, D)
        vdd = (U * d[None, :]) @ U.conj().T
        vdd = 0.5 * (vdd + vdd.conj().T)
        lam_min = float(d.min())
        n_aux = n_mt + n_ipw
        vt = np.zeros((n_aux, n_aux), dtype=np.complex128)
        # index of every dense-block member in the (a,L,M,P') + IPW ordering
        dense_idx = np.empty(D, dtype=np.int64)
        for a in range(n_at):
            for lm in range(nlm_aux):
                dense_idx[a * nlm_aux + lm] = (a * nlm_aux + lm) * P
        dense_idx[n_at * nlm_aux:] = n_mt + np.arange(n_ipw)
        vt[np.ix_(dense_idx, dense_idx)] = vdd
        if P > 1:
            for a in range(n_at):
                for lm in range(nlm_aux):
                    base = (a * nlm_aux + lm) * P
                    L = int(math.isqrt(lm))
                    kap = rng.uniform(0.0, gp_max)
                    w = _cn(rng, (P - 1, P - 1))
                    bc = s * 4.0 * math.pi / (kap * kap + 0.05) * 0.5 * (
                        np.eye(P - 1) + w @ w.conj().T / (P - 1))
                    bc = 0.5 * (bc + bc.conj().T)
                    cc = _cn(rng, (P - 1,))
                    q = float(np.real(cc.conj() @ np.linalg.solve(bc, cc)))
                    cc = cc * math.sqrt(0.25 * lam_min / q)
                    vt[base + 1:base + P, base + 1:base + P] = bc
                    vt[base + 1:base + P, base] = cc
                    vt[base, base + 1:base + P] = cc.conj()
        # back to the original basis: v = Q^T v_t Q with Q block-diagonal, one
        # frame per (a,L,M) block of the MT rows and the identity on the IPW
        # rows; applied block by block (rows, then columns)
        Fb = np.stack([frames[a][int(math.isqrt(lm))] for a in range(n_at) for lm in range(nlm_aux)])
        nblk = Fb.shape[0]
        vq = vt.copy()
        vq[:n_mt] = np.einsum("bji,bjc->bic", Fb, vq[:n_mt].reshape(nblk, P, n_aux)).reshape(n_mt, n_aux)
        vq[:, :n_mt] = np.einsum("rbj,bji->rbi", vq[:, :n_mt].reshape(n_aux, nblk, P), Fb).reshape(n_aux, n_mt)
        v.append(0.5 * (vq + vq.conj().T))

    return System(name=str(spec["name"]), lattice=lattice, pos_frac=pos, rmt=rmt, lmax=lmax,
                  Lmax=Lmax, P=P, mesh=mesh_t, gmax=float(spec["gmax"]), n_bands=n_bands,
                  n_occ=n_occ, Gk=Gk, c=c, A=A, R=R, mu=mu, Gaux=Gaux, v=v, sparse=sparse,
                  scale=s, seed=seed)


def _make_system_inv(cfg, *, seed=None, mesh=None, nb=None, no=None, aux=None, scale=None) -> System:
    """The inversion-symmetric variant of a workload (module docstring)."""
    if isinstance(cfg, int):
        index = cfg
        spec = dict(CONFIGS[cfg])
    else:
        index = 99
        spec = dict(cfg)
    for key, val in (("mesh", mesh), ("nb", nb), ("no", no), ("aux", aux), ("scale", scale)):
        if val is not None:
            spec[key] = val
    if seed is None:
        seed = SEED_BASE + 100 + index
    rng = np.random.Generator(np.random.PCG64(seed))

    lattice = np.asarray(spec["lattice"], dtype=np.float64)
    pos = np.asarray(spec.get("pos_inv", spec["pos"]), dtype=np.float64)
    rmt = np.asarray(spec["rmt"], dtype=np.float64)
    mesh_t = tuple(int(x) for x in spec["mesh"])
    n_k = int(np.prod(mesh_t))
    n_at = pos.shape[0]
    lmax, Lmax, P = int(spec["lmax"]), int(spec["Lmax"]), int(spec["P"])
    n_lmp = 2 * (lmax + 1) ** 2
    n_lp = 2 * (lmax + 1)
    nlm_aux = (Lmax + 1) ** 2
    if sphere_gap(lattice, pos, rmt) <= 0.0:
        raise ValueError("muffin-tin spheres overlap")
    partner = inversion_partners(pos, rmt)

    def draw(spec_val):
        if isinstance(spec_val, tuple):
            return rng.integers(spec_val[1], spec_val[2] + 1, size=n_k)
        return np.full(n_k, int(spec_val))
    n_bands = draw(spec["nb"]).astype(np.int32)
    n_occ = np.minimum(draw(spec["no"]).astype(np.int32), n_bands)

    a_scale = float(spec.get("a_scale", 1.0))
    Gk, c, A = [], [], []
    for ik in range(n_k):
        kf = kpoint_frac(mesh_t, ik)
        g, _ = _g_sphere(kf, lattice, float(spec["gmax"]))
        Gk.append(g)
        npw = g.shape[0]
        nbk = int(n_bands[ik])
        c.append(rng.standard_normal((nbk, npw)).astype(np.complex128) / math.sqrt(npw))
        Ak = np.zeros((nbk, n_at, n_lmp), dtype=np.complex128)
        for a in range(n_at):
            b = int(partner[a])
            if b < a:
                continue
            ph = np.exp(2j * math.pi * float(kf @ (pos[a] + pos[b])))   # e^{ik.T_a}
            for l in range(lmax + 1):
                for m in range(-l, l + 1):
                    for p in range(2):
                        i, j = 2 * (l * l + l + m) + p, 2 * (l * l + l - m) + p
                        sg = 1.0 if (l + m) % 2 == 0 else -1.0
                        if b != a:
                            Ak[:, a, i] = _cn(rng, nbk) * a_scale
                            Ak[:, b, j] = sg * ph * np.conj(Ak[:, a, i])
                        elif m > 0:
                            Ak[:, a, i] = _cn(rng, nbk) * a_scale
                            Ak[:, a, j] = sg * ph * np.conj(Ak[:, a, i])
                        elif m == 0:
                            x = rng.standard_normal(nbk) * a_scale / math.sqrt(2.0)
                            Ak[:, a, i] = np.exp(1j * math.pi * float(kf @ (pos[a] + pos[b]))) * (
                                x if l % 2 == 0 else 1j * x)
        A.append(Ak)

    R = rng.standard_normal((n_at, (Lmax + 1) * P, n_lp, n_lp)) * 0.1
    R = np.triu(R) + np.swapaxes(np.triu(R, 1), -1, -2)
    mu = rng.standard_normal((n_at, (Lmax + 1) * P))
    for a in range(n_at):
        if partner[a] < a:
            R[a] = R[partner[a]]
            mu[a] = mu[partner[a]]

    aux_spec = spec["aux"]
    Gaux, gnorm = [], []
    if aux_spec[0] == "count":
        counts = rng.integers(aux_spec[1], aux_spec[2] + 1, size=n_k)
    for iq in range(n_k):
        qf = kpoint_frac(mesh_t, iq)
        if aux_spec[0] == "cut":
            g, nrm = _g_sphere(qf, lattice, float(aux_spec[1]))
        else:
            g, nrm = _g_count(qf, lattice, int(counts[iq]))
        Gaux.append(g)
        gnorm.append(nrm)
    gp_max = max(float(x.max()) if x.size else 0.0 for x in gnorm)

    s = float(spec["scale"])
    sparse = bool(spec["sparse"])
    n_mt = n_at * nlm_aux * P

    def second(a, L, M):
        """(a, L, M) is the second function of its pair: its channel copies the first's."""
        b = int(partner[a])
        return (b < a) or (b == a and M > 0)

    frames = None
    if sparse:
        frames = [[_frame_with_first_row(rng, mu[a, L * P:(L + 1) * P]) for L in range(Lmax + 1)]
                  for a in range(n_at)]
        for a in range(n_at):
            if partner[a] < a:
                frames[a] = frames[partner[a]]
    v = []
    for iq in range(n_k):
        n_ipw = Gaux[iq].shape[0]
        if not sparse:
            n = n_mt + n_ipw
            kappa = rng.uniform(0.0, gp_max, size=n_mt)
            g = np.concatenate([kappa, gnorm[iq]])
            d = s * 4.0 * math.pi / (g * g + 0.05)
            O = _haar_orthogonal(rng, n)
            vq = (O * d[None, :]) @ O.T
            v.append((0.5 * (vq + vq.T)).astype(np.complex128))
            continue
        D = n_at * nlm_aux + n_ipw
        kappa = rng.uniform(0.0, gp_max, size=n_at * nlm_aux)
        g = np.concatenate([kappa, gnorm[iq]])
        d = s * 4.0 * math.pi / (g * g + 0.05)
        O = _haar_orthogonal(rng, D)
        vdd = (O * d[None, :]) @ O.T
        vdd = 0.5 * (vdd + vdd.T)
        lam_min = float(d.min())
        n_aux = n_mt + n_ipw
        vt = np.zeros((n_aux, n_aux), dtype=np.float64)
        dense_idx = np.empty(D, dtype=np.int64)
        for a in range(n_at):
            for lm in range(nlm_aux):
                dense_idx[a * nlm_aux + lm] = (a * nlm_aux + lm) * P
        dense_idx[n_at * nlm_aux:] = n_mt + np.arange(n_ipw)
        vt[np.ix_(dense_idx, dense_idx)] = vdd
        if P > 1:
            blocks = {}
            for a in range(n_at):
                for L in range(Lmax + 1):
                    for M in range(-L, L + 1):
                        if second(a, L, M):
                            continue
                        kap = rng.uniform(0.0, gp_max)
                        w = rng.standard_normal((P - 1, P - 1))
                        bc = s * 4.0 * math.pi / (kap * kap + 0.05) * 0.5 * (np.eye(P - 1) + w @ w.T / (P - 1))
                        bc = 0.5 * (bc + bc.T)
                        cc = rng.standard_normal(P - 1)
                        q = float(cc @ np.linalg.solve(bc, cc))
                        cc = cc * math.sqrt(0.25 * lam_min / q)
                        blocks[(a, L, M)] = (bc, cc)
            for a in range(n_at):
                for L in range(Lmax + 1):
                    for M in range(-L, L + 1):
                        key = (int(partner[a]), L, -M) if second(a, L, M) else (a, L, M)
                        bc, cc = blocks[key]
                        base = (a * nlm_aux + L * L + L + M) * P
                        vt[base + 1:base + P, base + 1:base + P] = bc
                        vt[base + 1:base + P, base] = cc
                        vt[base, base + 1:base + P] = cc
        Fb = np.stack([frames[a][int(math.isqrt(lm))] for a in range(n_at) for lm in range(nlm_aux)])
        nblk = Fb.shape[0]
        vq = vt.copy()
        vq[:n_mt] = np.einsum("bji,bjc->bic", Fb, vq[:n_mt].reshape(nblk, P, n_aux)).reshape(n_mt, n_aux)
        vq[:, :n_mt] = np.einsum("rbj,bji->rbi", vq[:, :n_mt].reshape(n_aux, nblk, P), Fb).reshape(n_aux, n_mt)
        v.append((0.5 * (vq + vq.T)).astype(np.complex128))

    return System(name=str(spec["name"]) + "_inv", lattice=lattice, pos_frac=pos, rmt=rmt, lmax=lmax,
                  Lmax=Lmax, P=P, mesh=mesh_t, gmax=float(spec["gmax"]), n_bands=n_bands,
                  n_occ=n_occ, Gk=Gk, c=c, A=A, R=R, mu=mu, Gaux=Gaux, v=v, sparse=sparse,
                  scale=s, seed=seed, inversion=True)


def radial_grid(rmt: float, n_r: int):
    """Gauss-Legendre nodes and weights on (0, rmt] for int_0^rmt g(r) dr."""
    x, w = np.polynomial.legendre.leggauss(int(n_r))
    return 0.5 * rmt * (x + 1.0), 0.5 * rmt * w


def radial_functions(lmax: int, rmt: float, n_r: int, seed: int):
    """Seeded stand-ins for the LAPW radial functions u_lp(r) of one atom
    (p = 0: the solution, p = 1: its energy derivative, Eq. FLAPW-basis): smooth
    functions r^l (a_0 + a_1 r + ... + a_4 r^4) with random coefficients on the
    Gauss-Legendre grid of radial_grid.  Returns (r, w, u[2(lmax+1)][n_r])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r, w = radial_grid(rmt, n_r)
    u = np.zeros((2 * (lmax + 1), r.size))
    for l in range(lmax + 1):
        for p in range(2):
            a = rng.standard_normal(5) / (1.0 + np.arange(5)) ** 2
            x = r / rmt
            u[2 * l + p] = x ** l * (a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3 + a[4] * x ** 4)
    return r, w, u


def coulomb_dense_block(sysm, iq: int, seed: Optional[int] = None) -> np.ndarray:
    """A seeded Hermitian positive-definite stand-in for the dense block of the
    transformed Coulomb matrix of Fig. 1 (the functions with a multipole, one per
    (a, L, M) in the MT order, then the interstitial plane waves of q):
    U diag(s 4 pi / (g^2 + 0.05)) U^H with g = |q + G| for the plane waves and
    U(0, max|q+G|) for the MT functions, U Haar-unitary."""
    rng = np.random.Generator(np.random.PCG64((sysm.seed if seed is None else seed) * 1000 + 900 + iq))
    B = reciprocal(sysm.lattice)
    qf = kpoint_frac(sysm.mesh, iq)
    gn = np.linalg.norm((qf[None, :] + sysm.Gaux[iq]) @ B, axis=1)
    nch = sysm.n_atoms * (sysm.Lmax + 1) ** 2
    kappa = rng.uniform(0.0, float(gn.max()) if gn.size else 1.0, size=nch)
    g = np.concatenate([kappa, gn])
    d = sysm.scale * 4.0 * math.pi / (g * g + 0.05)
    U = _haar_unitary(rng, g.size)
    v = (U * d[None, :]) @ U.conj().T
    return 0.5 * (v + v.conj().T)
