"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: textbook
closed forms, independent numerical quadrature, brute-force real-space
integrals, invariances and identities stated in Sec. III of the paper.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as integrate
import scipy.special as sp

from oracle import oracle as O
from paper_1003_0524_gb300 import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(cfg=1, **kw):
    base = dict(mesh=(2, 2, 2), nb=3, no=2)
    base.update(kw)
    return S.make_system(cfg, **base)


# --------------------------------------------------------------- Gaunt

def test_threej_closed_forms():
    rows = np.loadtxt(os.path.join(GOLDEN, "threej_closed_forms.txt"))
    for r in rows:
        j1, j2, j3, m1, m2, m3 = (int(x) for x in r[:6])
        assert O.threej(j1, j2, j3, m1, m2, m3) == pytest.approx(r[6], abs=1e-15)


def _sphere_quad(nth=16, nph=32):
    x, w = np.polynomial.legendre.leggauss(nth)
    th = np.arccos(x)
    ph = np.arange(nph) * 2 * math.pi / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = np.outer(w, np.full(nph, 2 * math.pi / nph))
    return TH, PH, W


def test_gaunt_vs_quadrature_and_selection_rules():
    """G(LM;lm;l'm') = int Y*_LM Y*_lm Y_l'm' against scipy's spherical
    harmonics on a quadrature exact for the degrees involved (<= 12)."""
    TH, PH, W = _sphere_quad()
    Y = {}
    for l in range(5):
        for m in range(-l, l + 1):
            Y[(l, m)] = sp.sph_harm_y(l, m, TH, PH)
    worst = 0.0
    for L in range(5):
        for M in range(-L, L + 1):
            for l1 in range(5):
                for m1 in range(-l1, l1 + 1):
                    for l2 in range(5):
                        for m2 in range(-l2, l2 + 1):
                            g = O.gaunt(L, M, l1, m1, l2, m2)
                            allowed = (m2 == m1 + M and abs(l1 - l2) <= L <= l1 + l2
                                       and (L + l1 + l2) % 2 == 0)
                            if not allowed:
                                assert g == 0.0
                                continue
                            q = np.sum(W * np.conj(Y[(L, M)]) * np.conj(Y[(l1, m1)]) * Y[(l2, m2)])
                            assert abs(q.imag) < 1e-14
                            worst = max(worst, abs(q.real - g))
    assert worst < 1e-14


def test_gaunt_monopole():
    for l in range(5):
        for m in range(-l, l + 1):
            assert O.gaunt(0, 0, l, m, l, m) == pytest.approx(1.0 / (2.0 * math.sqrt(math.pi)), abs=1e-15)


# ------------------------------------------------------- step function

def test_theta_zero_is_interstitial_fraction():
    s = S.make_system(0)
    o = O.Oracle(s)
    expect = 1.0 - 4.0 * math.pi * 2.2 ** 3 / 3.0 / 512.0
    assert o.theta([[0, 0, 0]])[0] == pytest.approx(expect, abs=1e-15)
    assert expect == pytest.approx(0.912886253709833, abs=1e-12)


def test_theta_vs_radial_quadrature():
    """Theta_K = -(1/Omega) sum_a e^{-iK.R_a} int_sphere e^{-iK.s} d^3s for K != 0,
    with the sphere integral done numerically as 4 pi int_0^S s^2 sin(Ks)/(Ks) ds."""
    s = _tiny(1)
    o = O.Oracle(s)
    B = s.recip()
    om = abs(np.linalg.det(s.lattice))
    for K in ([1, 0, 0], [1, 1, 0], [2, -1, 1], [0, 3, -2]):
        kc = np.asarray(K) @ B
        kn = np.linalg.norm(kc)
        tot = 0.0j
        for a in range(s.n_atoms):
            S_a = s.rmt[a]
            rad, _ = integrate.quad(lambda r: r * r * math.sin(kn * r) / (kn * r), 0.0, S_a,
                                    epsabs=1e-15, epsrel=1e-13)
            ra = s.pos_frac[a] @ s.lattice
            tot += np.exp(-1j * kc @ ra) * 4 * math.pi * rad
        assert o.theta([K])[0] == pytest.approx(-tot / om, abs=1e-13)


def _inside_any_sphere(pts_cart, s):
    inside = np.zeros(pts_cart.shape[0], bool)
    shifts = np.stack(np.meshgrid(*[np.arange(-1, 2)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for a in range(s.n_atoms):
        for t in shifts:
            c = (s.pos_frac[a] + t) @ s.lattice
            inside |= np.sum((pts_cart - c) ** 2, axis=1) < s.rmt[a] ** 2
    return inside


def test_zipw_real_space_brute_force_single_plane_waves():
    """<M_G^q phi_m,k-q | phi_n,k> with single plane-wave bands, integrated on a
    fine real-space grid with Theta(r) evaluated pointwise.  Pins the step
    function, the sign of every reciprocal vector in the Theta index and the
    umklapp vector G0 of the pair."""
    s = _tiny(1, nb=1, no=1)
    # pick a pair whose k - q needs folding (G0 != 0)
    ik, iq = 1 * 4 + 0 * 2 + 1, 1 * 4 + 1 * 2 + 1   # k=(1,0,1)/2, q=(1,1,1)/2
    o0 = O.Oracle(s)
    ikp, G0 = o0.fold(ik, iq)
    assert np.any(G0 != 0)
    # single plane waves: band 0 of k has only its 3rd PW, band 0 of k' its 5th
    ia, ib = 4, 2
    for kk, idx in ((ikp, ia), (ik, ib)):
        c = np.zeros_like(s.c[kk])
        c[0, idx] = 1.0
        s.c[kk] = c
    o = O.Oracle(s)
    Z = o.zipw(ik, iq)[:, 0, 0]
    Ga, Gb = s.Gk[ikp][ia], s.Gk[ik][ib]
    B = s.recip()
    n = 72
    f = (np.arange(n) + 0.5) / n
    F = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    R = F @ s.lattice
    theta = ~_inside_any_sphere(R, s)
    om = abs(np.linalg.det(s.lattice))
    kf, qf, kpf = s.kpoint_frac(ik), s.kpoint_frac(iq), s.kpoint_frac(ikp)
    for g in range(0, s.Gaux[iq].shape[0], 7):
        G = s.Gaux[iq][g]
        wv = (-(qf + G) - (kpf + Ga) + (kf + Gb)) @ B
        val = np.sum(theta * np.exp(1j * R @ wv)) * om / n ** 3 / om ** 1.5
        # the grid sum converges like 1/n; 2e-3 of Theta_0 is far below the
        # difference between neighbouring Theta_K
        assert abs(val - Z[g]) < 2e-3 / math.sqrt(om), (g, val, Z[g])
    # the opposite umklapp sign gives a visibly different value
    K_wrong = s.Gaux[iq][0] + Ga - Gb + G0
    K_right = s.Gaux[iq][0] + Ga - Gb - G0
    assert abs(o.theta([K_wrong])[0] - o.theta([K_right])[0]) > 1e-2


def test_zipw_two_step_equals_direct_triple_sum():
    s = S.make_system(0, nb=3, no=2)
    o = O.Oracle(s)
    for ik, iq in ((0, 0), (3, 5), (7, 1)):
        a = o.zipw(ik, iq)
        b = o.zipw(ik, iq, direct=True)
        assert np.abs(a - b).max() < 1e-15 * max(1.0, np.abs(b).max()) * 50


def test_zipw_no_spheres_is_plain_convolution():
    """With S_a -> 0 the step function is 1 everywhere (Theta_K = delta_K0) and
    Z^IPW reduces to Omega^{-1/2} sum_G1 conj(c_G1(m)) c_{G+G1-G0}(n)."""
    s = _tiny(1)
    s.rmt = np.zeros_like(s.rmt)
    o = O.Oracle(s)
    ik, iq = 5, 3
    ikp, G0 = o.fold(ik, iq)
    Z = o.zipw(ik, iq)
    idx = {tuple(g): i for i, g in enumerate(s.Gk[ik])}
    om = abs(np.linalg.det(s.lattice))
    for g, G in enumerate(s.Gaux[iq]):
        ref = np.zeros((Z.shape[1], Z.shape[2]), complex)
        for i1, G1 in enumerate(s.Gk[ikp]):
            j = idx.get(tuple(G + G1 - G0))
            if j is not None:
                ref += np.outer(np.conj(s.c[ikp][:, i1]), s.c[ik][:, j])[: Z.shape[1]]
        assert np.abs(Z[g] - ref / math.sqrt(om)).max() < 1e-15


# ------------------------------------------------------------- Z^MT

def test_zmt_three_dimensional_quadrature():
    """Z^MT against a brute-force 3-D quadrature of
    int_sphere conj(M^q_aLMP(r)) conj(phi_m,k'(r)) phi_n,k(r) d^3r
    with explicit polynomial radial functions u_lp and M_LP, the MT Bloch
    function of Eq. (MT functions) restricted to the home cell and the
    wave functions of Eq. (FLAPW-basis) inside the sphere."""
    s = _tiny(1)
    lmax, Lmax, P = s.lmax, s.Lmax, s.P
    rng = np.random.default_rng(7)
    alpha = rng.uniform(-0.3, 0.3, (s.n_atoms, lmax + 1, 2))
    gam = rng.uniform(-0.3, 0.3, (s.n_atoms, Lmax + 1, P))

    def u(a, l, p, r):
        return r ** l * (1.0 + alpha[a, l, p] * r) * (0.5 + 0.1 * p)

    def Mrad(a, L, Pi, r):
        return r ** L * (0.3 + gam[a, L, Pi] * r ** (Pi + 1))

    xr, wr = np.polynomial.legendre.leggauss(16)
    R = np.zeros_like(s.R)
    for a in range(s.n_atoms):
        Sa = s.rmt[a]
        r = 0.5 * Sa * (xr + 1.0)
        w = 0.5 * Sa * wr
        for L in range(Lmax + 1):
            for Pi in range(P):
                for l in range(lmax + 1):
                    for p in range(2):
                        for l2 in range(lmax + 1):
                            for p2 in range(2):
                                R[a, L * P + Pi, 2 * l + p, 2 * l2 + p2] = np.sum(
                                    w * r * r * Mrad(a, L, Pi, r) * u(a, l, p, r) * u(a, l2, p2, r))
    s.R = R
    o = O.Oracle(s)
    ik, iq = 6, 3
    ikp, _ = o.fold(ik, iq)
    Z = o.zmt(ik, iq)
    TH, PH, W = _sphere_quad(14, 28)
    Y = {(l, m): sp.sph_harm_y(l, m, TH, PH) for l in range(max(lmax, Lmax) + 1)
         for m in range(-l, l + 1)}
    qc = s.kpoint_frac(iq) @ s.recip()
    nlm = (Lmax + 1) ** 2
    for a in range(s.n_atoms):
        Sa = s.rmt[a]
        r = 0.5 * Sa * (xr + 1.0)
        wrad = 0.5 * Sa * wr * r * r
        ra = s.pos_frac[a] @ s.lattice
        bloch = np.exp(1j * qc @ ra)  # M^q in the home cell: M(r - R_a) e^{i q.R_a}

        def phi(Acoef, n):
            out = np.zeros((r.size,) + TH.shape, complex)
            for l in range(lmax + 1):
                for m in range(-l, l + 1):
                    for p in range(2):
                        cidx = 2 * (l * l + l + m) + p
                        out += (Acoef[n, a, cidx] * u(a, l, p, r)[:, None, None]
                                * Y[(l, m)][None])
            return out

        phim = [phi(s.A[ikp], m) for m in range(Z.shape[1])]
        phin = [phi(s.A[ik], n) for n in range(Z.shape[2])]
        for L in range(Lmax + 1):
            for M in range(-L, L + 1):
                for Pi in range(P):
                    I = (a * nlm + L * L + L + M) * P + Pi
                    Mq = Mrad(a, L, Pi, r)[:, None, None] * Y[(L, M)][None] * bloch
                    for m in range(Z.shape[1]):
                        for n in range(Z.shape[2]):
                            integ = np.conj(Mq) * np.conj(phim[m]) * phin[n]
                            val = np.einsum("r,ij,rij->", wrad, W, integ)
                            assert abs(val - Z[I, m, n]) < 1e-12 * max(1.0, abs(val)), (I, m, n)


# -------------------------------------------------- multipole transform

def test_transform_orthogonal_and_multipole_free():
    rng = np.random.default_rng(3)
    for P in (1, 2, 3, 4, 6):
        for _ in range(5):
            mu = rng.standard_normal(P)
            T = O.transform_T(mu)
            assert np.abs(T @ T.T - np.eye(P)).max() < 1e-15 * 8
            tm = T @ mu
            assert tm[0] == pytest.approx(np.linalg.norm(mu), rel=1e-14)
            assert np.abs(tm[1:]).max(initial=0.0) < 1e-14 * np.linalg.norm(mu) * 4


def test_transform_two_functions_is_paper_formula():
    mu = np.array([0.7, -1.3])
    n = math.hypot(*mu)
    T = O.transform_T(mu)
    assert np.allclose(T, np.array([[mu[0], mu[1]], [mu[1], -mu[0]]]) / n, atol=1e-16, rtol=0)


def test_vx_invariant_under_transform_and_sparse_pattern():
    """V^x(dense v, Z) = V^x(T v T^T, T Z) (the transform is orthogonal), and
    the generator's v becomes block-sparse in the transformed basis: every
    element that couples a multipole-free function to anything outside its own
    (a, L, M) channel vanishes (Fig. 1)."""
    s = _tiny(1, nb=4, no=2)
    o = O.Oracle(s)
    for ik in (0, 5):
        V = o.vx(ik, q0term=False)
        Vt = o.vx(ik, transformed=True, q0term=False)
        assert np.abs(V - Vt).max() < 1e-12 * np.abs(V).max()
    P, nlm = s.P, (s.Lmax + 1) ** 2
    Tfull = np.eye(s.n_aux(0))
    for a in range(s.n_atoms):
        for L in range(s.Lmax + 1):
            T = O.transform_T(s.mu[a, L * P:(L + 1) * P])
            for M in range(-L, L + 1):
                b = (a * nlm + L * L + L + M) * P
                Tfull[b:b + P, b:b + P] = T
    vt = Tfull @ s.v[0] @ Tfull.T
    scale = np.abs(vt).max()
    for a in range(s.n_atoms):
        for lm in range(nlm):
            b = (a * nlm + lm) * P
            for i in range(1, P):
                row = vt[b + i].copy()
                row[b:b + P] = 0.0
                assert np.abs(row).max() < 1e-13 * scale


# ----------------------------------------------------------------- V^x

def _literal_vx(s, o, ik):
    """Literal four-index sum of Eq. (vec-mat-vec) with numpy."""
    nb = int(s.n_bands[ik])
    V = np.zeros((nb, nb), complex)
    for iq in range(s.n_k):
        Z = o.z(ik, iq)  # (I, m, n)
        V -= np.einsum("imn,ij,jmp->np", np.conj(Z), s.v[iq], Z)
    return V / s.n_k


def test_vx_hermitian_nsd_and_literal_sum():
    s = _tiny(1, nb=4, no=2)
    o = O.Oracle(s)
    for ik in (0, 3, 6):
        V = o.vx(ik, q0term=False)
        assert np.abs(V - V.conj().T).max() < 1e-14 * np.abs(V).max()
        ev = np.linalg.eigvalsh(0.5 * (V + V.conj().T))
        assert ev.max() < 1e-14 * np.abs(ev).max()
        L = _literal_vx(s, o, ik)
        assert np.abs(V - L).max() < 1e-13 * np.abs(L).max()


def test_vx_linear_in_v():
    s = _tiny(1, nb=3, no=2)
    o1 = O.Oracle(s)
    V1 = o1.vx(2, q0term=False)
    s.v = [2.0 * v for v in s.v]
    o2 = O.Oracle(s)
    V2 = o2.vx(2, q0term=False)
    assert np.abs(V2 - 2 * V1).max() < 1e-14 * np.abs(V2).max()


# ---------------------------------------------------------------- q->0

def test_q0_constants():
    beta = 0.005  # Sec. III.E: beta = 0.005, e^{-beta q0^2} = beta
    q0 = math.sqrt(-math.log(beta) / beta)
    assert math.exp(-beta * q0 * q0) == pytest.approx(beta, rel=1e-14)
    assert q0 == pytest.approx(32.5519, abs=1e-3)


def test_q0_analytic_integral():
    """(1/2pi^2) int_{|q|<q0} e^{-beta q^2}/q^2 d^3q = (pi beta)^{-1/2} erf(sqrt(beta) q0)."""
    beta = 0.005
    q0 = math.sqrt(-math.log(beta) / beta)
    num, _ = integrate.quad(lambda q: 4 * math.pi * math.exp(-beta * q * q), 0.0, q0,
                            epsabs=1e-14, epsrel=1e-14)
    assert num / (2 * math.pi ** 2) == pytest.approx(
        math.erf(math.sqrt(beta) * q0) / math.sqrt(math.pi * beta), rel=1e-13)


def test_q0_bracket_vanishes_with_mesh_density():
    """The bracket of Eq. (div final) is the integral minus its Riemann sum
    without the q=0 cell, so it goes to 0 like N_k^{-1/3}; this pins the
    4 pi / (N_k Omega) weight of the discrete sum."""
    vals = []
    for n in (2, 4, 8):
        s = S.make_system(0, mesh=(n, n, n), nb=1, no=1)
        vals.append(O.Oracle(s).vdiv())
    assert vals[0] > vals[1] > vals[2] > 0
    assert vals[2] / vals[1] == pytest.approx(0.5, abs=0.08)
    assert vals[1] / vals[0] == pytest.approx(0.5, abs=0.12)


def test_q0_term_on_occupied_diagonal_only():
    s = _tiny(1, nb=4, no=2)
    o = O.Oracle(s)
    d = o.vx(1, q0term=True) - o.vx(1, q0term=False)
    b = o.vdiv()
    no = int(s.n_occ[1])
    expect = np.zeros_like(d)
    expect[np.arange(no), np.arange(no)] = -b
    assert np.abs(d - expect).max() < 1e-13


# ---------------------------------------------------------------- E_x

def test_exchange_energy_identity():
    """E_x = (1/2)(1/N_k) sum_k sum_n f_nk V_nn(k) equals the double sum
    -(1/2)(1/N_k^2) sum_{k,q} sum_{n occ(k), m occ(k-q)} Z^H v Z of
    Eq. (HF exchange energy), and is negative for positive-definite v."""
    s = _tiny(1, nb=4, no=2)
    o = O.Oracle(s)
    V = {ik: o.vx(ik, q0term=False) for ik in range(s.n_k)}
    ex = O.exchange_energy(s, V)
    dbl = 0.0
    for ik in range(s.n_k):
        no = int(s.n_occ[ik])
        for iq in range(s.n_k):
            Z = o.z(ik, iq)[:, :, :no]
            dbl += np.real(np.einsum("imn,ij,jmn->", np.conj(Z), s.v[iq], Z))
    dbl *= -0.5 / s.n_k ** 2
    assert ex == pytest.approx(dbl, rel=1e-13)
    assert ex < 0


# ---------------------------------------------------------------- LAPW representation (Eq. APW trafo)

def _hpd(rng, n):
    w = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2)
    s = np.eye(n) + 0.3 * (w @ w.conj().T) / n
    return 0.5 * (s + s.conj().T)


def _s_orthonormal(rng, S, nb):
    """Coefficients c (rows: bands) with c* S c^T = 1, i.e. <phi_n|phi_n'> = delta."""
    ev, U = np.linalg.eigh(S)
    s_inv_half = (U / np.sqrt(ev)) @ U.conj().T
    z = rng.standard_normal((S.shape[0], nb)) + 1j * rng.standard_normal((S.shape[0], nb))
    q, _ = np.linalg.qr(z)
    return (s_inv_half @ q).T


def test_lapw_trafo_round_trip_recovers_band_matrix():
    """With a square S-orthonormal coefficient matrix the transform is the
    change of basis c^{-H} V c^{-1}; projecting back with the coefficients,
    c* V_GG' c^T, must give V again (Eq. APW trafo, Sec. III.A)."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 9
    S = _hpd(rng, n)
    c = _s_orthonormal(rng, S, n)
    assert np.abs(c.conj() @ S @ c.T - np.eye(n)).max() < 1e-12
    V = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    V = V + V.conj().T
    Vgg = O.lapw_trafo(S, c, V)
    assert np.abs(c.conj() @ Vgg @ c.T - V).max() < 1e-11 * np.abs(V).max()
    assert np.abs(Vgg - Vgg.conj().T).max() < 1e-12 * np.abs(Vgg).max()


def test_lapw_trafo_of_unit_band_matrix_is_a_projector():
    """For fewer bands than basis functions and V = 1, S^{-1} V_GG' is the
    S-orthogonal projector onto the span of the bands: idempotent, with trace
    equal to the number of bands."""
    rng = np.random.Generator(np.random.PCG64(12))
    npw, nb = 14, 5
    S = _hpd(rng, npw)
    c = _s_orthonormal(rng, S, nb)
    Vgg = O.lapw_trafo(S, c, np.eye(nb))
    Pm = np.linalg.solve(S, Vgg)
    assert np.abs(Pm @ Pm - Pm).max() < 1e-12
    assert abs(np.trace(Pm) - nb) < 1e-12


# ---------------------------------------------------------------- k.p term at q = 0 (Appendix A)

def _antiherm(rng, nb):
    w = rng.standard_normal((3, nb, nb)) + 1j * rng.standard_normal((3, nb, nb))
    return 0.5 * (w - np.conj(np.swapaxes(w, 1, 2)))


def test_kp_term_two_band_closed_form():
    """Two bands, the lower occupied, p_x = [[0, x], [-x*, 0]] (and y, z alike):
    D_10 = -i p_10 / (e_0 - e_1), so Abar_00 = -(4 pi/3) s and Abar_11 = +(4 pi/3) s with
    s = sum_a |x_a|^2 / (e_1 - e_0)^2, and Abar_01 = 0; the term added to V^x is
    -Abar / (N_k Omega)."""
    x = np.array([0.3 + 0.1j, -0.2j, 0.05])
    p = np.zeros((3, 2, 2), np.complex128)
    p[:, 0, 1] = x
    p[:, 1, 0] = -np.conj(x)
    e = np.array([-0.5, 0.7])
    nko = 123.0
    t = O.kp_term(e, p, 1, nko)
    s = float(np.sum(np.abs(x) ** 2)) / (e[1] - e[0]) ** 2
    c = 4.0 * np.pi / 3.0 * s / nko
    assert abs(t[0, 0] - c) < 1e-15 and abs(t[1, 1] + c) < 1e-15
    assert abs(t[0, 1]) < 1e-18 and abs(t[1, 0]) < 1e-18


def test_kp_term_vanishes_with_every_band_occupied_and_is_hermitian():
    """D is anti-Hermitian (p is), so D D^H = D^H D: with every band of the
    window occupied the two sums of the occupied-occupied case cancel.  With
    some bands empty the term is Hermitian and its empty-empty block is
    negative semi-definite (minus a Gram matrix)."""
    rng = np.random.Generator(np.random.PCG64(21))
    nb = 7
    e = np.sort(rng.uniform(-1, 1, nb))
    p = _antiherm(rng, nb)
    assert np.abs(O.kp_term(e, p, nb, 10.0)).max() < 1e-13
    t = O.kp_term(e, p, 3, 10.0)
    assert np.abs(t - t.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(t[3:, 3:]).max() < 1e-14
    assert np.abs(O.kp_term(e, 2 * p, 3, 10.0) - 4 * t).max() < 1e-13   # quadratic in p
    assert np.abs(O.kp_term(e + 0.37, p, 3, 10.0) - t).max() < 1e-13   # only energy differences


def test_kp_term_skips_degenerate_pairs():
    """First-order k.p does not fix the mixing inside a degenerate pair: such
    pairs contribute nothing (no division by a zero energy difference)."""
    rng = np.random.Generator(np.random.PCG64(22))
    e = np.array([-1.0, -0.5, 0.4, 0.4, 1.0])
    p = _antiherm(rng, 5)
    t = O.kp_term(e, p, 2, 10.0)
    assert np.all(np.isfinite(t))
    p2 = p.copy()
    p2[:, 2, 3] = 0.0
    p2[:, 3, 2] = 0.0
    assert np.abs(O.kp_term(e, p2, 2, 10.0) - t).max() < 1e-15
