"""The MT product basis and on-site Coulomb blocks built on the GPU from radial
functions (Sec. III.B-C), against the FP64 oracle (GB300 only).

hfx_set_radial_functions builds, per atom, the product functions M_aLP
(linear-dependence removal, constant function for L = 0), their multipole
moments, the radial integrals R and the on-site Coulomb blocks C.  With
HFX_LAYOUT_TRANSFORMED_ONSITE the caller gives only the part of v_t that
involves the functions with a multipole; the library fills the rows and
columns of the multipole-free functions from C.  The oracle builds the same
basis itself and assembles the whole v(q) in the original basis from its own
C and multipole transform.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1003_0524_gb300 import hfx
from paper_1003_0524_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1003_0524_gb300 import build
    build.build()
    hfx.load()


def _radial(s, a, n_r=300):
    return S.radial_functions(s.lmax, float(s.rmt[a]), n_r, seed=s.seed * 10 + a)


@pytest.mark.parametrize("cfg", [1, 4])
def test_radial_basis_matches_oracle(cfg):
    s = S.make_system(cfg, mesh=(1, 1, 2), nb=4, no=2, **({"aux": ("count", 100, 100)} if cfg >= 3 else {}))
    with hfx.Context(s, precision="sliced") as c:
        for a in range(s.n_atoms):
            r, w, u = _radial(s, a)
            hfx.hfx_set_radial_functions(c.ctx, a, r, w, u, 1e-4)
            got = hfx.hfx_get_radial_basis(c.ctx, a, r.size, s.lmax, s.Lmax, s.P)
            ref = O.mpb_radial(r, w, u, s.lmax, s.Lmax, s.P, 1e-4)
            for key in ("M", "mu", "R", "C"):
                err = np.abs(got[key] - ref[key]).max()
                assert err <= 1e-10 * max(1.0, np.abs(ref[key]).max()), (a, key, err)


def test_too_few_product_functions_is_rejected():
    s = S.make_system(1, mesh=(1, 1, 2), nb=4, no=2)
    r, w = S.radial_grid(float(s.rmt[0]), 200)
    # every u_lp the same function: one product per L, fewer than P = 3
    u = np.stack([r * 0 + 1.0 + r for _ in range(2 * (s.lmax + 1))])
    with hfx.Context(s, precision="sliced") as c:
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_radial_functions(c.ctx, 0, r, w, u, 1e-4)
        assert e.value.code == hfx.HFX_EINVAL


def _onsite_case(cfg, **kw):
    s = S.make_system(cfg, **kw)
    P, nlm = s.P, (s.Lmax + 1) ** 2
    rad = [_radial(s, a) for a in range(s.n_atoms)]
    basis = [O.mpb_radial(r, w, u, s.lmax, s.Lmax, P, 1e-4) for (r, w, u) in rad]
    # what the caller gives: the dense block (functions with a multipole, and the
    # plane waves) in the transformed index positions, zero elsewhere
    v_lib, v_ora = [], []
    T = [[O.transform_T(basis[a]["mu"][L * P:(L + 1) * P]) for L in range(s.Lmax + 1)] for a in range(s.n_atoms)]
    for iq in range(s.n_k):
        nipw = s.Gaux[iq].shape[0]
        naux = s.n_mt + nipw
        vdd = S.coulomb_dense_block(s, iq)
        dense_idx = np.concatenate([np.arange(s.n_atoms * nlm) * P, s.n_mt + np.arange(nipw)])
        vt = np.zeros((naux, naux), np.complex128)
        vt[np.ix_(dense_idx, dense_idx)] = vdd
        v_lib.append(vt.copy())
        # the oracle's whole v_t: the multipole-free rows and columns from its C and T
        for a in range(s.n_atoms):
            for lm in range(nlm):
                L = int(np.sqrt(lm) + 1e-9)
                ch = (a * nlm + lm) * P
                blk = T[a][L] @ basis[a]["C"][L] @ T[a][L].T
                keep00 = vt[ch, ch]
                vt[ch:ch + P, ch:ch + P] = blk
                vt[ch, ch] = keep00
        # back to the original basis: v = T^T v_t T channel by channel
        Tb = np.zeros((naux, naux))
        for a in range(s.n_atoms):
            for lm in range(nlm):
                L = int(np.sqrt(lm) + 1e-9)
                ch = (a * nlm + lm) * P
                Tb[ch:ch + P, ch:ch + P] = T[a][L]
        Tb[s.n_mt:, s.n_mt:] = np.eye(nipw)
        vo = Tb.T @ vt @ Tb
        v_ora.append(0.5 * (vo + vo.conj().T))
    R = np.stack([b["R"] for b in basis])
    mu = np.stack([b["mu"] for b in basis])
    import dataclasses
    s_ora = dataclasses.replace(s, R=R, mu=mu, v=v_ora)
    return s, s_ora, rad, v_lib


@pytest.mark.parametrize("precision", ["fp64", "sliced"])
def test_onsite_layout_matches_oracle(precision):
    s, s_ora, rad, v_lib = _onsite_case(1, mesh=(2, 1, 2), nb=12, no=4)
    o = O.Oracle(s_ora)
    ref = {ik: o.vx(ik) for ik in range(s.n_k)}
    with hfx.Context(s, precision=precision) as c:
        for a, (r, w, u) in enumerate(rad):
            hfx.hfx_set_radial_functions(c.ctx, a, r, w, u, 1e-4)
        c.set_kpoints()
        for iq in range(s.n_k):
            hfx.hfx_set_coulomb(c.ctx, iq, s.Gaux[iq], v_lib[iq], layout=hfx.HFX_LAYOUT_TRANSFORMED_ONSITE)
        st = c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
    assert st["sparse_used"] == 1
    err = max(np.abs(V[k] - ref[k]).max() for k in ref)
    vmax = max(np.abs(ref[k]).max() for k in ref)
    print(f"onsite {precision}: max|dV| = {err:.3e} (max|V| {vmax:.3f})")
    if precision == "fp64":
        assert err <= 1e-10 * vmax
    else:
        assert err <= 1e-8
