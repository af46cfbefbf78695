"""Pins of the oracle's inversion-symmetric basis (Sec. III.D).

The symmetrized MT functions of Eqs. (sym MT functions) are defined by one
property: f(-r) = f(r)^*.  These tests evaluate the Bloch MT functions and the
wave functions in real space (scipy's spherical harmonics, explicit lattice
sums) and check that property point by point, then check its consequences:
real projection vectors, a real symmetric Coulomb matrix in the new basis,
and a V^x that the real arithmetic of the new basis reproduces.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import oracle as O
from paper_1003_0524_gb300 import synthetic as S


def _inv(cfg, **kw):
    base = dict(mesh=(2, 1, 2), nb=6, no=3)
    if cfg >= 3:
        base["aux"] = ("count", 150, 150)
    base.update(kw)
    return S.make_system(cfg, inversion=True, **base)


def _ylm(L, M, x):
    r = np.linalg.norm(x)
    th = math.acos(max(-1.0, min(1.0, x[2] / r)))
    ph = math.atan2(x[1], x[0])
    return complex(sp.sph_harm_y(L, M, th, ph))


def _radial(x, L, P, S_a):
    # any radial shape serves; partners use the same one (same species)
    return x ** L * (1.0 + 0.3 * (P + 1) * x) * (S_a - x)


def _bloch_mt(sysm, q_frac, r):
    """Every Bloch MT function M^q_(a,L,M,P)(r) of Eq. (MT functions) at the
    cartesian point r, in the oracle's (a, L, M, P) order."""
    lat = np.asarray(sysm.lattice)
    B = S.reciprocal(lat)
    q = q_frac @ B
    P = sysm.P
    out = np.zeros(sysm.n_mt, np.complex128)
    shifts = np.stack(np.meshgrid(*[np.arange(-2, 3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    nlm = (sysm.Lmax + 1) ** 2
    for a in range(sysm.n_atoms):
        Ra = sysm.pos_frac[a] @ lat
        for t in shifts:
            T = t @ lat
            x = r - T - Ra
            d = np.linalg.norm(x)
            if d >= sysm.rmt[a] or d < 1e-9:
                continue
            ph = np.exp(1j * float(q @ (T + Ra)))
            for L in range(sysm.Lmax + 1):
                for M in range(-L, L + 1):
                    y = _ylm(L, M, x)
                    for p in range(P):
                        out[(a * nlm + L * L + L + M) * P + p] += _radial(d, L, p, sysm.rmt[a]) * y * ph
    return out


def _points_in_spheres(sysm, rng, n):
    lat = np.asarray(sysm.lattice)
    pts = []
    for _ in range(n):
        a = int(rng.integers(sysm.n_atoms))
        t = rng.integers(-1, 2, size=3)
        u = rng.standard_normal(3)
        u *= rng.uniform(0.2, 0.9) * sysm.rmt[a] / np.linalg.norm(u)
        pts.append((sysm.pos_frac[a] + t) @ lat + u)
    return pts


@pytest.mark.parametrize("cfg", [0, 1, 3, 4])
def test_partners_and_unitary_S(cfg):
    s = _inv(cfg)
    ora = O.Oracle(s)
    p = ora.inv_partner()
    assert np.array_equal(p, S.inversion_partners(s.pos_frac, s.rmt))
    assert np.array_equal(p[p], np.arange(s.n_atoms))
    Sm = ora.sym_matrix()
    assert np.abs(Sm.conj().T @ Sm - np.eye(s.n_mt)).max() < 1e-14
    # at most two original functions per symmetrized one
    assert ((np.abs(Sm) > 0).sum(axis=0) <= 2).all()


@pytest.mark.parametrize("cfg", [0, 1, 3, 4])
def test_symmetrized_mt_functions_obey_f_minus_r_eq_conj(cfg):
    """Eqs. (sym MT functions) and the M = 0 rule: every column of S is a
    function with f(-r) = f(r)^*, at points inside the spheres, for a q that
    is not a reciprocal lattice vector."""
    s = _inv(cfg)
    Sm = O.Oracle(s).sym_matrix()
    rng = np.random.default_rng(11 + cfg)
    q = np.array([0.25, 0.5, -0.25])
    worst, scale = 0.0, 0.0
    for r in _points_in_spheres(s, rng, 6):
        fp = Sm.T @ _bloch_mt(s, q, r)
        fm = Sm.T @ _bloch_mt(s, q, -r)
        worst = max(worst, float(np.abs(fm - fp.conj()).max()))
        scale = max(scale, float(np.abs(fp).max()))
    assert scale > 0.1
    assert worst < 1e-12 * scale
    # the original functions do not have the property (the test has teeth)
    r = _points_in_spheres(s, rng, 1)[0]
    m0, m1 = _bloch_mt(s, q, r), _bloch_mt(s, q, -r)
    assert np.abs(m1 - m0.conj()).max() > 1e-3 * np.abs(m0).max()


@pytest.mark.parametrize("cfg", [0, 1, 3, 4])
def test_generated_wave_functions_obey_psi_minus_r_eq_conj(cfg):
    """The generator's inversion variant: real plane-wave coefficients, and MT
    coefficients with psi(-r) = psi(r)^* inside the spheres, where
    psi(R_a + T + x) = e^{ik.T} sum_lmp A^a_lmp u_lp(|x|) Y_lm(x)."""
    s = _inv(cfg)
    lat = np.asarray(s.lattice)
    B = S.reciprocal(lat)
    rng = np.random.default_rng(5 + cfg)
    for ik in range(s.n_k):
        assert np.abs(s.c[ik].imag).max() == 0.0
        k = s.kpoint_frac(ik) @ B
        A = s.A[ik]

        def psi(r, n):
            for a in range(s.n_atoms):
                for t in np.stack(np.meshgrid(*[np.arange(-2, 3)] * 3, indexing="ij"), -1).reshape(-1, 3):
                    T = t @ lat
                    x = r - T - s.pos_frac[a] @ lat
                    d = np.linalg.norm(x)
                    if d < s.rmt[a]:
                        acc = 0j
                        for l in range(s.lmax + 1):
                            for m in range(-l, l + 1):
                                y = _ylm(l, m, x)
                                for p in range(2):
                                    acc += A[n, a, 2 * (l * l + l + m) + p] * d ** l * (1 + 0.5 * p * d) * y
                        return np.exp(1j * float(k @ T)) * acc
            raise AssertionError("point outside every sphere")

        for r in _points_in_spheres(s, rng, 3):
            for n in (0, A.shape[0] - 1):
                a, b = psi(r, n), psi(-r, n)
                assert abs(b - np.conj(a)) < 1e-12 * max(1.0, abs(a))


def _zsym(ora, s, Sm, ik, iq):
    Zmt = ora.zmt(ik, iq)
    Zs = np.einsum("ij,imn->jmn", Sm.conj(), Zmt)       # Z' = S^H Z
    return np.concatenate([Zs, ora.zipw(ik, iq)], axis=0)


@pytest.mark.parametrize("cfg", [0, 1, 3, 4])
def test_projections_are_real_in_the_symmetrized_basis(cfg):
    s = _inv(cfg)
    ora = O.Oracle(s)
    Sm = ora.sym_matrix()
    for ik, iq in ((0, 1), (s.n_k - 1, s.n_k - 2), (1, 0)):
        Z = _zsym(ora, s, Sm, ik, iq)
        assert np.abs(Z.imag).max() < 1e-12 * np.abs(Z).max()
        # in the original basis the MT rows are complex
        assert np.abs(ora.zmt(ik, iq).imag).max() > 1e-3 * np.abs(Z).max()


def test_broken_symmetry_gives_complex_projections():
    """A planted mistake in one MT coefficient of the partner atom shows up as
    an imaginary part of Z' (the reality check is not vacuous)."""
    s = _inv(1)
    s.A[0] = s.A[0].copy()
    s.A[0][0, 1, 2 * (1 * 1 + 1 + 1)] *= 1j
    ora = O.Oracle(s)
    Z = _zsym(ora, s, ora.sym_matrix(), 0, 1)
    assert np.abs(Z.imag).max() > 1e-4 * np.abs(Z).max()


@pytest.mark.parametrize("cfg", [0, 1, 4])
def test_vx_from_the_real_form_matches_the_complex_oracle(cfg):
    """Eq. (vec-mat-vec) in the symmetrized basis, in real arithmetic
    (V = -(1/N_k) sum_q sum_m Z'^T v' Z', v' the given real matrix), equals
    the oracle's complex V^x with v = S v' S^H; V^x is real symmetric."""
    s = _inv(cfg)
    ora = O.Oracle(s)
    Sm = ora.sym_matrix()
    for vq in s.v:
        assert np.abs(vq.imag).max() == 0.0
        assert np.abs(vq - vq.T).max() == 0.0
    ik = s.n_k - 1
    nb = int(s.n_bands[ik])
    Vr = np.zeros((nb, nb))
    for iq in range(s.n_k):
        Z = _zsym(ora, s, Sm, ik, iq).real
        Vr -= np.einsum("imn,ij,jmp->np", Z, s.v[iq].real, Z) / s.n_k
    Vc = ora.vx(ik, q0term=False)
    assert np.abs(Vc.imag).max() < 1e-12 * np.abs(Vc).max()
    assert np.abs(Vc.real - Vr).max() < 1e-12 * np.abs(Vc).max()
    assert np.abs(Vr - Vr.T).max() < 1e-12 * np.abs(Vr).max()
