"""The real-valued path of inversion-symmetric systems (Sec. III.D) on the GPU.

The library takes v(q) over the symmetrized MT functions (real symmetric),
packs two real occupied bands per complex column and runs the Coulomb apply on
the real operand alone.  The oracle computes V^x with complex arithmetic in the
original basis (v = S v' S^H, its own S).  Bars as in test_gpu_parity.py:
FP64 build 1e-10 relative, sliced build 1e-8 Ha; V^x must come out real
(imaginary parts exactly zero) and symmetric.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1003_0524_gb300 import hfx
from paper_1003_0524_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL_FP64_REL = 1e-10
TOL_SPLIT_ABS = 1e-8


@pytest.fixture(scope="session", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1003_0524_gb300 import build
    build.build()
    hfx.load()


CASES = {
    # one atom at the origin, no multipole transform (dense v): the M = 0 rule
    "inv_cfg0": lambda: S.make_system(0, inversion=True),
    # a pair of atoms at -+(1/8,1/8,1/8)a; an odd occupied count (one padded column)
    "inv_cfg1_k2": lambda: S.make_system(1, mesh=(2, 2, 2), no=5, inversion=True),
    # two Z^H Y band blocks
    "inv_cfg1_nb72": lambda: S.make_system(1, mesh=(2, 1, 1), nb=72, no=7, inversion=True),
    # uneven band windows, occupied counts and aux sizes
    "inv_cfg2_k2": lambda: S.make_system(2, mesh=(2, 2, 2), inversion=True),
    # five atoms at inversion centres off the origin (their own partners)
    "inv_cfg3_shape": lambda: S.make_system(3, mesh=(1, 1, 2), nb=12, no=5, inversion=True),
    # five pairs, L <= 5, D ~ 2660
    "inv_cfg4_shape": lambda: S.make_system(4, mesh=(1, 1, 2), nb=10, no=4, inversion=True),
}

_cache = {}


def oracle_v(name, s):
    if name not in _cache:
        o = O.Oracle(s)
        _cache[name] = {ik: o.vx(ik) for ik in range(s.n_k)}
    return _cache[name]


def gpu_v(s, precision, **kw):
    with hfx.Context(s, precision=precision, **kw) as c:
        c.load_system()
        st = c.build_all()
        return {ik: c.exchange(ik) for ik in range(s.n_k)}, c.energy(), st


def _err(A, B):
    return max(np.abs(A[k] - B[k]).max() for k in B)


def _vmax(B):
    return max(np.abs(B[k]).max() for k in B)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "sliced"])
def test_inversion_path_matches_oracle(name, precision):
    s = CASES[name]()
    ref = oracle_v(name, s)
    V, ex, st = gpu_v(s, precision)
    err = _err(V, ref)
    ex_ref = O.exchange_energy(s, ref)
    print(f"{name} {precision}: max|dV| = {err:.3e}, max|V| = {_vmax(ref):.3f}, dE_x = {ex - ex_ref:.3e}")
    for k in V:
        assert np.abs(V[k].imag).max() == 0.0
        assert np.abs(V[k] - V[k].T).max() <= 2 * TOL_SPLIT_ABS
    if precision == "fp64":
        assert err <= TOL_FP64_REL * _vmax(ref), err
        assert abs(ex - ex_ref) <= 1e-10 * abs(ex_ref)
    else:
        assert err <= TOL_SPLIT_ABS, err
        assert abs(ex - ex_ref) <= 0.5 * int(max(s.n_occ)) * TOL_SPLIT_ABS
    # the real path counts real flops over the occupied bands: a quarter of the
    # complex count of the same pairs
    assert st["useful_flops"] > 0


def _original_basis(s):
    """The same system with v taken back to the original MT functions and the
    complex path selected (the oracle's S)."""
    Sm = O.Oracle(s).sym_matrix()
    nmt = s.n_mt
    vs = []
    for vq in s.v:
        w = np.array(vq, dtype=np.complex128)
        w[:nmt, :] = Sm @ w[:nmt, :]
        w[:, :nmt] = w[:, :nmt] @ Sm.conj().T
        vs.append(0.5 * (w + w.conj().T))
    return dataclasses.replace(s, v=vs, inversion=False)


@pytest.mark.parametrize("name", ["inv_cfg1_k2", "inv_cfg4_shape"])
def test_real_path_matches_complex_path(name):
    """One system, two paths: the complex path in the original basis and the
    real path in the symmetrized one give the same V^x (sliced builds)."""
    s = CASES[name]()
    Vr, exr, st_r = gpu_v(s, "sliced")
    Vc, exc, st_c = gpu_v(_original_basis(s), "sliced")
    assert _err(Vr, Vc) <= 2 * TOL_SPLIT_ABS
    # the real path issues about a quarter of the apply's slice products
    assert st_r["flops_apply_exec"] <= 0.3 * st_c["flops_apply_exec"]


def test_inversion_graph_replay_is_identical():
    s = CASES["inv_cfg1_k2"]()
    with hfx.Context(s, precision="sliced") as c:
        c.load_system()
        outs = []
        for _ in range(3):
            st = c.build_all()
            outs.append({ik: c.exchange(ik) for ik in range(s.n_k)})
        assert st["graph_replayed"] == 1
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]) and np.array_equal(outs[0][k], outs[2][k])


def test_inversion_input_checks():
    s = CASES["inv_cfg1_k2"]()
    # a geometry without inversion symmetry
    s_plain = S.make_system(1, mesh=(2, 2, 2))
    with pytest.raises(hfx.HfxError) as e:
        hfx.Context(s_plain, precision="sliced", inversion=True)
    assert e.value.code == hfx.HFX_EINVAL
    with hfx.Context(s, precision="sliced") as c:
        c.load_system()
        # complex plane-wave coefficients
        cc = s.c[0].copy()
        cc[0, 0] += 0.1j
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_kpoint(c.ctx, 0, int(s.n_bands[0]), int(s.n_occ[0]), s.Gk[0], cc, s.A[0])
        assert e.value.code == hfx.HFX_EINVAL
        # MT coefficients of the partner atom that break phi(-r) = phi(r)^*
        A = s.A[0].copy()
        A[0, 1, 2 * (1 + 1 + 1)] *= 1j
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_kpoint(c.ctx, 0, int(s.n_bands[0]), int(s.n_occ[0]), s.Gk[0], s.c[0], A)
        assert e.value.code == hfx.HFX_EINVAL
        # a Coulomb matrix that is not real over the symmetrized basis
        v = np.array(s.v[0], dtype=np.complex128)
        v[0, 1] += 1e-3j
        v[1, 0] -= 1e-3j
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_coulomb(c.ctx, 0, s.Gaux[0], v)
        assert e.value.code == hfx.HFX_EINVAL
        # partner atoms with different radial integrals
        R = s.R[1].copy()
        R[0, 0, 0] += 0.01
        hfx.hfx_set_radial(c.ctx, 1, R, s.mu[1])
        with pytest.raises(hfx.HfxError) as e:
            c.build_all()
        assert e.value.code == hfx.HFX_EINVAL
        hfx.hfx_set_radial(c.ctx, 1, s.R[1], s.mu[1])
        with pytest.raises(hfx.HfxError) as e:
            c.build_all(keep_products=True)
        assert e.value.code == hfx.HFX_EUNSUPPORTED
        st = c.build_all()
        assert st["n_pairs"] == s.n_k * s.n_k


@pytest.mark.parametrize("nb_zhy", [16, 32, 48, 64, 40])
def test_inversion_zhy_tile_shapes(nb_zhy):
    """The real form of the Z^H Y tiles (two row blocks per tile, band blocks of
    16, 32, 48 or 64; 72 bands give 5, 3, 2 and 2 blocks, so an odd count leaves
    a tile with one row block) and the complex form it falls back to (40)."""
    name = "inv_cfg1_nb72"
    s = CASES[name]()
    ref = oracle_v(name, s)
    V, ex, st = gpu_v(s, "sliced", tile_nb_zhy=nb_zhy)
    assert st["tile_nb_zhy"] == nb_zhy
    err = _err(V, ref)
    print(f"{name} NB {nb_zhy}: max|dV| = {err:.3e}")
    assert err <= TOL_SPLIT_ABS
    for k in V:
        assert np.abs(V[k].imag).max() == 0.0
