"""Pins of the oracle's MT product basis and on-site Coulomb integrals (Sec. III.B-C).

The radial Coulomb integral is pinned by closed forms for power functions; the
product basis by orthonormality, the constant function of L = 0, the rank of a
set of products that are linearly dependent by construction, and the Coulomb
self-energy of the constant function (a uniformly charged sphere).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1003_0524_gb300 import synthetic as S


def _closed(a, b, L, Sr):
    """4 pi/(2L+1) int int r^a r'^b r<^L/r>^(L+1) r^2 r'^2 over [0, S]^2, a, b >= L."""
    first = Sr ** (a + b + 5) / ((b + L + 3) * (a + b + 5))
    second = (Sr ** (b + 2 - L) * Sr ** (a + L + 3) / (a + L + 3) - Sr ** (a + b + 5) / (a + b + 5)) / (b + 2 - L)
    return 4 * math.pi / (2 * L + 1) * (first + second)


@pytest.mark.parametrize("L", [0, 1, 2, 4, 5])
def test_radial_coulomb_closed_forms(L):
    Sr = 2.2
    r, w = S.radial_grid(Sr, 1500)
    for a, b in ((L, L), (L, L + 2), (L + 1, L + 3)):
        v = O.radial_coulomb(r, w, L, r ** a, r ** b)
        ref = _closed(a, b, L, Sr)
        assert abs(v - ref) <= 2e-6 * abs(ref), (a, b, v, ref)
        # symmetric kernel
        assert abs(v - O.radial_coulomb(r, w, L, r ** b, r ** a)) <= 1e-13 * abs(v)


def test_radial_coulomb_converges_with_the_grid():
    Sr, L = 1.8, 1
    errs = []
    for n in (100, 200, 400):
        r, w = S.radial_grid(Sr, n)
        errs.append(abs(O.radial_coulomb(r, w, L, r, r) - _closed(1, 1, L, Sr)))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


def test_product_basis_orthonormal_constant_and_coulomb():
    Sr, lmax, Lmax, P = 2.2, 4, 4, 3
    r, w, u = S.radial_functions(lmax, Sr, 600, seed=7)
    b = O.mpb_radial(r, w, u, lmax, Lmax, P)
    M, mu, R, C = b["M"], b["mu"], b["R"], b["C"]
    for L in range(Lmax + 1):
        G = (M[L * P:(L + 1) * P] * (w * r * r)) @ M[L * P:(L + 1) * P].T
        assert np.abs(G - np.eye(P)).max() < 1e-12
        assert np.abs(C[L] - C[L].T).max() < 1e-12 * np.abs(C[L]).max()
        assert np.linalg.eigvalsh(C[L]).min() > 0.0       # the Coulomb kernel is positive definite
    c = math.sqrt(3.0 / Sr ** 3)
    assert np.abs(M[0] - c).max() < 1e-12
    assert abs(mu[0] - c * Sr ** 3 / 3) < 1e-12
    # a uniformly charged sphere: 4 pi c^2 * 2 S^5 / 15
    assert abs(C[0, 0, 0] - 8 * math.pi * Sr ** 2 / 5) < 1e-5 * C[0, 0, 0]
    assert np.abs(R - np.swapaxes(R, 1, 2)).max() < 1e-14
    # R is the radial integral of the definition
    i = 1 * P + 2
    assert abs(R[i, 3, 6] - np.sum(w * r * r * M[i] * u[3] * u[6])) < 1e-14


def test_linear_dependence_removal_keeps_the_rank():
    """u_lp = r^l (1 + p r), l <= 2: the L = 0 products r^(2l) (1 + p r)(1 + p' r)
    span the polynomials of degree <= 6 (rank 7; 6 after the constant), so
    P = 7 works and P = 8 finds too few functions above the threshold."""
    Sr, lmax = 2.0, 2
    r, w = S.radial_grid(Sr, 200)
    u = np.stack([r ** l * (1 + p * r) for l in range(lmax + 1) for p in range(2)])
    b = O.mpb_radial(r, w, u, lmax, 0, 7, thr=1e-10)
    # the kept functions span r^3: its projection onto them is complete
    x = r ** 3
    coef = (b["M"] * (w * r * r)) @ x
    res = x - coef @ b["M"]
    assert np.sqrt(np.sum(w * r * r * res ** 2)) < 1e-8 * np.sqrt(np.sum(w * r * r * x ** 2))
    with pytest.raises(ValueError):
        O.mpb_radial(r, w, u, lmax, 0, 8, thr=1e-10)


def test_product_basis_at_the_papers_lmax():
    """lmax = 8 (the paper's setting for its crystals): 171 candidate products per
    L; the kept functions stay orthonormal and their Coulomb blocks positive
    definite."""
    Sr, lmax, Lmax, P = 2.1, 8, 4, 4
    r, w, u = S.radial_functions(lmax, Sr, 300, seed=11)
    b = O.mpb_radial(r, w, u, lmax, Lmax, P)
    for L in range(Lmax + 1):
        M = b["M"][L * P:(L + 1) * P]
        G = (M * (w * r * r)) @ M.T
        assert np.abs(G - np.eye(P)).max() < 1e-10
        assert np.linalg.eigvalsh(b["C"][L]).min() > 0.0
