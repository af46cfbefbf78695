"""Parity of the CUDA library against the FP64 CPU oracle (GB300 only).

Every comparison goes through the C ABI (paper_1003_0524_gb300.hfx).  Bars:
  FP64 build      max|dV| <= 1e-10 * max|V|      (relative, FP64 arithmetic)
  sliced build    max|dV| <= 1e-8 Ha             (V scaled so that max|V_nn| ~ 1 Ha;
                                                  tensor-core fixed-point slices)
Projection vectors are compared part by part (MT, interstitial) because the
interstitial part is much smaller than the MT part in V.
"""
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


_cache = {}


def oracle_v(key, sysm, ks, q0=True):
    ck = (key, tuple(ks), q0)
    if ck not in _cache:
        o = O.Oracle(sysm)
        _cache[ck] = {ik: o.vx(ik, q0term=q0) for ik in ks}
    return _cache[ck]


def gpu_v(sysm, precision, ks=None, **kw):
    with hfx.Context(sysm, precision=precision, **kw) as c:
        c.load_system()
        st = c.build_all()
        ks = range(sysm.n_k) if ks is None else ks
        V = {ik: c.exchange(ik) for ik in ks}
        return V, c.energy(), st


def max_err(A, B):
    return max(np.abs(A[k] - B[k]).max() for k in B)


def vmax(B):
    return max(np.abs(B[k]).max() for k in B)


SMALL = {
    "cfg0": lambda: S.make_system(0),
    "cfg1_k2": lambda: S.make_system(1, mesh=(2, 2, 2)),
    "cfg2_k2": lambda: S.make_system(2, mesh=(2, 2, 2)),
    # several band blocks in every tensor-core stage (72 bands)
    "cfg1_nb72": lambda: S.make_system(1, mesh=(2, 1, 1), nb=72, no=6),
    # the cells, atoms, aux sizes and MT channels of configs 3 and 4 on a 1x1x2
    # mesh with narrow band windows, so that the oracle stays fast
    "cfg3_shape": lambda: S.make_system(3, mesh=(1, 1, 2), nb=12, no=4),
    "cfg4_shape": lambda: S.make_system(4, mesh=(1, 1, 2), nb=10, no=4),
    # the same cells with 72 bands: two Z^H Y band blocks, L <= 5 and the
    # dense block D ~ 2660 of config 4, D ~ 1225 of config 3
    "cfg3_nb72": lambda: S.make_system(3, mesh=(1, 1, 2), nb=72, no=8),
    "cfg4_nb72": lambda: S.make_system(4, mesh=(1, 1, 2), nb=72, no=8),
    # the literal MT coefficient distribution A ~ CN(0, 1) (a_scale 1): the MT
    # rows of Z (bilinear in A) then dwarf the interstitial rows of the same
    # column by ~240x.  v is scaled down so that max|V| stays ~ 1 Ha (with the
    # usual scale 24 max|V| is ~ 2.8e3 Ha on this case)
    "cfg1_ascale1": lambda: S.make_system(dict(S.CONFIGS[1], a_scale=1.0, scale=1.5e-3),
                                          mesh=(2, 2, 1), nb=8, no=4),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_fp64_matches_oracle(name):
    s = SMALL[name]()
    ref = oracle_v(name, s, range(s.n_k))
    V, ex, st = gpu_v(s, "fp64")
    err = max_err(V, ref)
    assert err <= TOL_FP64_REL * vmax(ref), (err, vmax(ref))
    assert st["sparse_used"] == (1 if s.sparse else 0)
    ex_ref = O.exchange_energy(s, ref)
    assert abs(ex - ex_ref) <= 1e-10 * abs(ex_ref)


@pytest.mark.parametrize("name", list(SMALL))
def test_split_matches_oracle(name):
    s = SMALL[name]()
    ref = oracle_v(name, s, range(s.n_k))
    V, ex, st = gpu_v(s, "sliced")
    err = max_err(V, ref)
    ex_ref = O.exchange_energy(s, ref)
    print(f"{name}: max|dV| = {err:.3e} Ha, max|V| = {vmax(ref):.3f}, dE_x = {ex - ex_ref:.3e}")
    assert err <= TOL_SPLIT_ABS, err
    for k in V:
        assert np.abs(V[k] - V[k].conj().T).max() <= 2 * TOL_SPLIT_ABS
    # E_x = (1/2)(1/N_k) sum_k sum_{n < n_occ} Re V_nn, so |dE_x| is at most
    # (1/2) max_k n_occ(k) times the bar on |dV|
    assert abs(ex - ex_ref) <= 0.5 * int(max(s.n_occ)) * TOL_SPLIT_ABS, ex - ex_ref


# In the sliced build every projection is a slice product: each operand line
# is kept to 2^-32 of its largest element, so one product over K terms is off
# by up to ~K 2^-32 of (largest |a|)(largest |b|).  Z^MT is one product
# (K = 50); Z^IPW is a product with T_n, which is itself a product of Theta
# and c (K ~ 500) and is re-sliced against the largest |T_n| of the whole box.
# Relative to the pair's largest projection, which is much smaller than those
# operand maxima, this gives a few 1e-9 (measured up to 5e-9 for Z^IPW, 1e-9
# for Z^MT); the bar is 1e-8.
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("sliced", 1e-8)])
def test_projections_match_oracle(precision, tol):
    s = S.make_system(1, mesh=(2, 2, 2), nb=6, no=3)
    o = O.Oracle(s)
    with hfx.Context(s, precision=precision) as c:
        c.load_system()
        c.build_all(keep_products=True)
        for ik, iq in ((0, 0), (3, 5), (7, 2), (5, 7)):
            ikp, _ = o.fold(ik, iq)
            Z = c.products(ik, iq, ikp)
            zm, zi = o.zmt(ik, iq), o.zipw(ik, iq)
            nmt = s.n_mt
            em = np.abs(Z[:nmt] - zm).max() / np.abs(zm).max()
            ei = np.abs(Z[nmt:] - zi).max() / np.abs(zi).max()
            print(f"{precision} Z ({ik},{iq}): MT rel {em:.2e}, IPW rel {ei:.2e}")
            assert em <= tol and ei <= tol


def test_q0_bracket_matches_oracle():
    """Both sides sum ~10^6 terms in FP64 in different orders, and the bracket
    is the difference of two numbers near 8 that cancel to ~0.14, so the
    agreement is bounded by ~1e-16 * 8 * sqrt(10^6) / 0.14 ~ 1e-11 relative."""
    s = S.make_system(1, mesh=(2, 2, 2), nb=2, no=1)
    with hfx.Context(s, precision="fp64") as c:
        b = c.q0_bracket()
    assert b == pytest.approx(O.Oracle(s).vdiv(), rel=1e-10)


def test_dense_and_sparse_forms_agree():
    s = S.make_system(1, mesh=(2, 2, 2), nb=8, no=4)
    Vs, _, sts = gpu_v(s, "fp64", sparse="on")
    Vd, _, std = gpu_v(s, "fp64", sparse="off")
    assert sts["sparse_used"] == 1 and std["sparse_used"] == 0
    assert max_err(Vs, Vd) <= 1e-11 * vmax(Vd)


def test_q0_term_off():
    s = S.make_system(0, nb=6, no=3)
    ref = oracle_v("cfg0_q0off", s, range(s.n_k), q0=False)
    V, _, _ = gpu_v(s, "fp64", q0_term=False)
    assert max_err(V, ref) <= TOL_FP64_REL * vmax(ref)


def test_build_exchange_single_k_matches_build_all():
    s = S.make_system(1, mesh=(2, 2, 2), nb=8, no=3)
    with hfx.Context(s, precision="sliced") as c:
        c.load_system()
        c.build_all()
        Vall = c.exchange(5)
        V5 = c.build_exchange(5)
    assert np.abs(Vall - V5).max() <= 1e-12 * np.abs(Vall).max()


def test_set_products_override():
    """Projection vectors supplied through the ABI replace the computed ones:
    with Z -> 2 Z for every pair, V^x (without the q->0 term) scales by 4."""
    s = S.make_system(0, nb=5, no=2)
    o = O.Oracle(s)
    ref = {ik: o.vx(ik, q0term=False) for ik in range(s.n_k)}
    with hfx.Context(s, precision="fp64", q0_term=False) as c:
        c.load_system()
        for ik in range(s.n_k):
            for iq in range(s.n_k):
                c.set_products(ik, iq, 2.0 * o.z(ik, iq))
        c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
        assert max(np.abs(V[k] - 4 * ref[k]).max() for k in ref) <= 1e-10 * vmax(ref)
        for ik in range(s.n_k):
            for iq in range(s.n_k):
                c.set_products(ik, iq, None)
        c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
        assert max_err(V, ref) <= 1e-10 * vmax(ref)


def test_edge_cases_empty_occupation_single_band_single_radial():
    """n_occ = 0 at some k (no m terms), one band, and P = 1 (no multipole-free
    functions, so the sparse form degenerates to the dense one)."""
    spec = dict(S.CONFIGS[0])
    spec["P"] = 1
    spec["name"] = "p1"
    s = S.make_system(spec, mesh=(2, 2, 1), nb=1, no=1)
    s.n_occ = s.n_occ.copy()
    s.n_occ[1] = 0
    o = O.Oracle(s)
    ref = {ik: o.vx(ik) for ik in range(s.n_k)}
    for prec, tol in (("fp64", TOL_FP64_REL * vmax(ref)), ("sliced", TOL_SPLIT_ABS)):
        V, _, _ = gpu_v(s, prec)
        assert max_err(V, ref) <= tol, prec


def test_error_paths():
    s = S.make_system(0, nb=3, no=2)
    with hfx.Context(s, precision="fp64") as c:
        with pytest.raises(hfx.HfxError) as e:
            c.build_all()
        assert e.value.code == hfx.HFX_EMISSING
        bad = s.v[0].copy()
        bad[0, 1] += 1.0
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_coulomb(c.ctx, 0, s.Gaux[0], bad)
        assert e.value.code == hfx.HFX_ENOTHERM
        nan = s.c[0].copy()
        nan[0, 0] = np.nan
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_kpoint(c.ctx, 0, int(s.n_bands[0]), int(s.n_occ[0]), s.Gk[0], nan, s.A[0])
        assert e.value.code == hfx.HFX_ENONFINITE
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_kpoint(c.ctx, 99, 1, 1, s.Gk[0], s.c[0], s.A[0])
        assert e.value.code == hfx.HFX_EINVAL
        Rb = s.R[0].copy()
        Rb[0, 0, 1] += 0.5
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_radial(c.ctx, 0, Rb, s.mu[0])
        assert e.value.code == hfx.HFX_EINVAL


def test_full_size_workload_sampled_k():
    """The benchmark workload (2-atom cell, 4x4x4 k, 40 bands, 8 occupied,
    N_aux ~ 635) in the launch configuration bench.py times: two sampled k
    points checked element by element against the oracle, every k checked for
    Hermiticity."""
    s = S.make_system(1)
    V, ex, st = gpu_v(s, "sliced")
    for ik in (0, 37):
        ref = O.Oracle(s).vx(ik)
        err = np.abs(V[ik] - ref).max()
        print(f"k={ik}: max|dV| = {err:.3e} Ha (max|V| = {np.abs(ref).max():.3f})")
        assert err <= TOL_SPLIT_ABS
    for k in V:
        assert np.abs(V[k] - V[k].conj().T).max() <= 2 * TOL_SPLIT_ABS
    assert st["n_pairs"] == 64 * 64


def test_many_batches_split_every_q():
    """A work budget far below the working set: the pairs are cut k-major into
    at least three batches, so the k points of every q fall into several
    batches (the path that configurations too large for one batch take)."""
    s = S.make_system(1, mesh=(2, 2, 2), nb=12, no=4)
    ref = oracle_v("cfg1_k2_nb12", s, range(s.n_k))
    for prec, tol in (("fp64", TOL_FP64_REL * vmax(ref)), ("sliced", TOL_SPLIT_ABS)):
        V, ex, st = gpu_v(s, prec, work_bytes=24 << 20)
        print(f"{prec}: {st['n_batches']} batches, max|dV| = {max_err(V, ref):.3e}")
        assert st["n_batches"] >= 3
        assert st["n_pairs"] == s.n_k * s.n_k
        assert max_err(V, ref) <= tol
        ex_ref = O.exchange_energy(s, ref)
        assert abs(ex - ex_ref) <= 0.5 * int(max(s.n_occ)) * tol


def test_graph_replay_is_identical():
    """The first build runs its launches directly, the second captures them as
    one CUDA graph and the third replays it: all three give the same bits, and
    so does a context that never captures."""
    s = S.make_system(1, mesh=(2, 2, 2), nb=10, no=4)
    with hfx.Context(s, precision="sliced") as c:
        c.load_system()
        runs = []
        for _ in range(3):
            st = c.build_all()
            runs.append(({ik: c.exchange(ik) for ik in range(s.n_k)}, st))
        assert runs[0][1]["graph_replayed"] == 0 and runs[2][1]["graph_replayed"] == 1
        assert runs[2][1]["n_launches"] == runs[0][1]["n_launches"]
        for V, _ in runs[1:]:
            for k in V:
                assert np.array_equal(V[k], runs[0][0][k])
    V2, _, st2 = gpu_v(s, "sliced", use_graph=False)
    for k in V2:
        assert np.array_equal(V2[k], runs[0][0][k])


def _transformed(c, s, v):
    """T v T^T with the context's own multipole transforms (Sec. III.C)."""
    nlm = (s.Lmax + 1) ** 2
    Q = np.eye(v.shape[0])
    for a in range(s.n_atoms):
        for L in range(s.Lmax + 1):
            T = hfx.hfx_get_transform(c.ctx, a, L, s.P)
            for M in range(2 * L + 1):
                b = (a * nlm + L * L + M) * s.P
                Q[b:b + s.P, b:b + s.P] = T
    return Q @ v @ Q.T


@pytest.mark.parametrize("precision", ["fp64", "sliced"])
def test_coulomb_given_transformed_matches_dense(precision):
    """hfx_set_coulomb with the layout TRANSFORMED (v_t = T v T^T, Fig. 1),
    passed with a row stride larger than N_aux, gives the V^x of the dense
    layout: 1e-12 relative in FP64, 1e-8 Ha in the sliced build."""
    s = S.make_system(1, mesh=(2, 2, 1), nb=8, no=3)
    Vd, _, _ = gpu_v(s, precision)
    with hfx.Context(s, precision=precision) as c:
        c.load_system(coulomb=False)
        for a in range(s.n_atoms):
            for L in range(s.Lmax + 1):
                T = hfx.hfx_get_transform(c.ctx, a, L, s.P)
                assert np.abs(T @ T.T - np.eye(s.P)).max() <= 1e-14
                mu = s.mu[a, L * s.P:(L + 1) * s.P]
                assert np.abs(T[0] - mu / np.linalg.norm(mu)).max() <= 1e-15
        for iq in range(s.n_k):
            vt = _transformed(c, s, s.v[iq])
            n = vt.shape[0]
            padded = np.zeros((n, n + 5), np.complex128)
            padded[:, :n] = vt
            hfx.hfx_set_coulomb(c.ctx, iq, s.Gaux[iq], padded, ld=n + 5, layout=hfx.HFX_LAYOUT_TRANSFORMED)
        st = c.build_all()
        assert st["sparse_used"] == 1
        Vt = {ik: c.exchange(ik) for ik in range(s.n_k)}
    tol = 1e-12 * vmax(Vd) if precision == "fp64" else TOL_SPLIT_ABS
    assert max_err(Vt, Vd) <= tol


def test_expired_device_wait_is_reported_and_recovered():
    """Failure detection without a GPU fault: the test hook makes one bounded
    wait of the Z^H Y kernel wait on a barrier that nothing completes.  The
    wait expires after about 1 ms, the kernel drains its copies and MMAs,
    frees its TMEM and returns; the build reports HFX_ETIMEOUT.  The next
    build on the same context is correct."""
    s = S.make_system(0, nb=6, no=3)
    ref = oracle_v("cfg0_nb6", s, range(s.n_k))
    with hfx.Context(s, precision="sliced", test_fail_wait=True) as c:
        c.load_system()
        with pytest.raises(hfx.HfxError) as e:
            c.build_all()
        assert e.value.code == hfx.HFX_ETIMEOUT
        c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
    assert max_err(V, ref) <= TOL_SPLIT_ABS


@pytest.mark.parametrize("nb_zhy,nb_zipw", [(8, 8), (24, 16), (48, 24), (56, 32), (64, 40), (40, 48), (16, 56),
                                            (64, 64)])
def test_tile_shapes_match_oracle(nb_zhy, nb_zipw):
    """Every band block the autotuner may choose for the Z^H Y tiles and for the
    interstitial tiles (both with K chunks of 64 up to 40 bands and of 32 above)
    gives the oracle's V^x within the bar, on 72 bands (several blocks, a ragged
    last one)."""
    s = SMALL["cfg1_nb72"]()
    ref = oracle_v("cfg1_nb72", s, range(s.n_k))
    V, _, st = gpu_v(s, "sliced", tile_nb_zhy=nb_zhy, tile_nb_zipw=nb_zipw)
    assert st["tile_nb_zhy"] == nb_zhy and st["tile_nb_zipw"] == nb_zipw
    assert max_err(V, ref) <= TOL_SPLIT_ABS


@pytest.mark.parametrize("precision", ["fp64", "sliced"])
def test_lapw_representation_matches_oracle(precision):
    """Eq. (APW trafo) on the GPU, V_GG'(k) = (S c) V^x (c^H S) for every k: against
    the oracle's transform of the same V^x (the transform alone, FP64, 1e-12
    relative), and against the oracle's transform of the oracle's V^x (end to
    end: the V^x bar carried through the two brackets)."""
    s = S.make_system(1, mesh=(2, 2, 1), nb=10, no=4)
    ref = oracle_v("cfg1_221_nb10", s, range(s.n_k))
    Sk = [S.overlap(s, ik) for ik in range(s.n_k)]
    with hfx.Context(s, precision=precision) as c:
        c.load_system()
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_lapw_transform_all(c.ctx)
        assert e.value.code == hfx.HFX_EMISSING
        c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
        bad = Sk[0].copy()
        bad[0, 1] += 0.5
        with pytest.raises(hfx.HfxError) as e:
            hfx.hfx_set_overlap(c.ctx, 0, bad)
        assert e.value.code == hfx.HFX_ENOTHERM
        for ik in range(s.n_k):
            hfx.hfx_set_overlap(c.ctx, ik, Sk[ik])
        st = hfx.hfx_lapw_transform_all(c.ctx)
        assert st["n_launches"] == 3
        Vg = {ik: hfx.hfx_get_lapw_exchange(c.ctx, ik, s.Gk[ik].shape[0]) for ik in range(s.n_k)}
    for ik in range(s.n_k):
        own = O.lapw_trafo(Sk[ik], s.c[ik], V[ik])
        assert np.abs(Vg[ik] - own).max() <= 1e-12 * np.abs(own).max()
        full = O.lapw_trafo(Sk[ik], s.c[ik], ref[ik])
        L = np.abs(Sk[ik] @ s.c[ik].T)            # |<chi_G|phi_n>|
        bound = float((L.sum(axis=1)[:, None] * L.sum(axis=1)[None, :]).max())
        tol = (TOL_FP64_REL * vmax(ref) if precision == "fp64" else TOL_SPLIT_ABS) * bound
        assert np.abs(Vg[ik] - full).max() <= tol
        assert np.abs(Vg[ik] - Vg[ik].conj().T).max() <= 1e-12 * np.abs(Vg[ik]).max() + tol


@pytest.mark.parametrize("precision", ["fp64", "sliced"])
def test_kp_term_matches_oracle(precision):
    """The k.p term at q = 0 (Appendix A) added in the build: V^x equals the
    oracle's V^x plus the oracle's term -Abar/(N_k Omega) of every k, at each
    build's bar; E_x follows from the diagonal.  Without hfx_set_momentum the
    build reports HFX_EMISSING."""
    s = S.make_system(1, mesh=(2, 2, 1), nb=10, no=4)
    ref = oracle_v("cfg1_221_nb10", s, range(s.n_k))
    o = O.Oracle(s)
    nko = s.n_k * o.omega()
    mom = [S.momentum(s, ik) for ik in range(s.n_k)]
    ref_kp = {ik: ref[ik] + O.kp_term(mom[ik][0], mom[ik][1], int(s.n_occ[ik]), nko) for ik in range(s.n_k)}
    with hfx.Context(s, precision=precision, kp_term=True) as c:
        c.load_system()
        with pytest.raises(hfx.HfxError) as e:
            c.build_all()
        assert e.value.code == hfx.HFX_EMISSING
        for ik in range(s.n_k):
            hfx.hfx_set_momentum(c.ctx, ik, *mom[ik])
        c.build_all()
        V = {ik: c.exchange(ik) for ik in range(s.n_k)}
        ex = c.energy()
    tol = TOL_FP64_REL * vmax(ref_kp) if precision == "fp64" else TOL_SPLIT_ABS
    assert max_err(V, ref_kp) <= tol
    assert max(np.abs(ref_kp[k] - ref[k]).max() for k in ref) > 100 * tol   # the term is visible
    ex_ref = O.exchange_energy(s, ref_kp)
    assert abs(ex - ex_ref) <= 0.5 * int(max(s.n_occ)) * tol
