"""The two largest workloads at their full sizes, in the launch configuration
bench.py times (GB300 only).

Config 3: 5-atom ABO3 cell, 6x6x6 k (46 656 pairs), 120 bands, N_aux = 1475.
Config 4: 10-atom corundum-like cell, 4x4x4 k (4096 pairs), 250 bands, N_aux = 3020,
and its inversion-symmetric variant (five atom pairs, real path of Sec. III.D).

The whole build runs through the C ABI.  The sampled sub-block V^x(k)[S][S]
(bands S: first and last occupied, first empty, last band) is compared element
by element with the FP64 oracle's values stored under tests/golden/ (written by
tests/golden/make_fullsize_samples.py, which calls only the oracle and the
input generator), and the whole V^x(k) of that k with the plain FP64 GPU build.
Every k is checked for Hermiticity.  Bar: 1e-8 Ha (max|V| ~ 1 Ha).
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_1003_0524_gb300 import hfx
from paper_1003_0524_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-8
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    spec = importlib.util.spec_from_file_location("make_fullsize_samples",
                                                  os.path.join(HERE, "golden", "make_fullsize_samples.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1003_0524_gb300 import build
    build.build()
    hfx.load()


@pytest.mark.parametrize("key", ["3", "4", "4inv"])
def test_full_size_sampled_block_matches_oracle(key):
    """4inv: the inversion-symmetric variant of config 4 on the real path
    (Sec. III.D); its V^x must also come out real."""
    g = _golden()
    seed, ik, bands, Vref = g.read(key)
    cfg, inv = g.SAMPLES[key][0], g.SAMPLES[key][1]
    s = S.make_system(cfg, inversion=inv)
    assert s.seed == seed
    with hfx.Context(s, precision="sliced") as c:
        c.load_system()
        st = c.build_all()
        V = {k: c.exchange(k) for k in range(s.n_k)}
    assert st["n_pairs"] == s.n_k * s.n_k
    Vs = V[ik][np.ix_(bands, bands)]
    err = float(np.abs(Vs - Vref).max())
    print(f"config {key}: {st['n_batches']} batches, {st['ms_total']:.0f} ms, "
          f"max|dV| vs oracle on k={ik} bands {bands}: {err:.3e} Ha (max|V| {np.abs(Vref).max():.3f})")
    assert err <= TOL
    for k in V:
        assert np.abs(V[k] - V[k].conj().T).max() <= 2 * TOL
        if inv:
            assert np.abs(V[k].imag).max() == 0.0
    # the plain FP64 GPU build of the same k (its N_k pairs)
    with hfx.Context(s, precision="fp64") as c64:
        c64.load_system()
        V64 = c64.build_exchange(ik)
    err64 = float(np.abs(V[ik] - V64).max())
    err64_ref = float(np.abs(V64[np.ix_(bands, bands)] - Vref).max())
    print(f"config {key}: max|dV| vs FP64 GPU on k={ik}: {err64:.3e} Ha; FP64 GPU vs oracle: {err64_ref:.3e}")
    assert err64 <= TOL
    assert err64_ref <= 1e-10 * np.abs(Vref).max()
