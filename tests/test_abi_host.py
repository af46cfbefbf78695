"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, exports every entry point that include/hfx.h declares, and the
Python binding refuses to run without it."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1003_0524_gb300 import build as B
from paper_1003_0524_gb300 import hfx
from paper_1003_0524_gb300 import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hfx.h")).read()
    return sorted(set(re.findall(r"HFX_API\s+[\w\s\*]*?\b(hfx_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_entry_points():
    names = _declared()
    assert "hfx_create" in names and "hfx_build_all" in names and "hfx_set_products" in names
    assert set(names) == set(hfx.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(hfx_\w+)", out))
    missing = set(_declared()) - exported
    assert not missing, missing
    # nothing but the C ABI leaks out of the library
    assert not {s for s in exported if not s.startswith("hfx_")}


def test_binding_loads_and_reports_status_strings(libpath):
    L = hfx.load()
    assert L.hfx_strerror(hfx.HFX_ENOTHERM).decode().startswith("Coulomb matrix")
    assert "sm_103a" in hfx.hfx_version()
    o = hfx.hfx_default_options()
    assert o.precision == hfx.HFX_PREC_SLICED and o.q0_term == 1 and o.beta == 0.005


def test_create_without_gpu_fails_cleanly(libpath):
    """On a machine without a usable GPU, hfx_create returns an error code
    (no crash, no silent CPU path)."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    s = S.make_system(0)
    with pytest.raises(hfx.HfxError) as e:
        hfx.Context(s)
    assert e.value.code in (hfx.HFX_EDEVICE, hfx.HFX_EUNSUPPORTED)


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(hfx, "_lib", None)
    monkeypatch.setattr(hfx, "library_path", lambda: str(tmp_path / "libhfx.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hfx.load()


def test_generator_is_deterministic_and_hermitian():
    a = S.make_system(0, nb=3, no=2)
    b = S.make_system(0, nb=3, no=2)
    for x, y in zip(a.c, b.c):
        assert np.array_equal(x, y)
    for v in a.v:
        assert np.abs(v - v.conj().T).max() < 1e-14 * np.abs(v).max()
        assert np.linalg.eigvalsh(v).min() > 0


def test_inversion_needs_partner_atoms(libpath):
    """hfx_create with inversion = 1 checks, before touching the device, that
    every atom has a partner at -R_a (same sphere radius): the zincblende pair
    of config 1 has none (HFX_EINVAL); the centred pair of its inversion
    variant passes the check and then needs the device."""
    plain = S.make_system(1, mesh=(1, 1, 2), nb=3, no=2)
    opt = hfx.hfx_default_options()
    opt.inversion = 1
    with pytest.raises(hfx.HfxError) as e:
        hfx.hfx_create(plain.lattice, plain.pos_frac, plain.rmt, plain.lmax, plain.Lmax, plain.P, plain.mesh, opt)
    assert e.value.code == hfx.HFX_EINVAL
    # unequal radii of the partners
    inv = S.make_system(1, mesh=(1, 1, 2), nb=3, no=2, inversion=True)
    with pytest.raises(hfx.HfxError) as e:
        hfx.hfx_create(inv.lattice, inv.pos_frac, np.array([2.2, 2.1]), inv.lmax, inv.Lmax, inv.P, inv.mesh, opt)
    assert e.value.code == hfx.HFX_EINVAL
    try:
        import torch
        if torch.cuda.is_available():
            return
    except ImportError:
        pass
    with pytest.raises(hfx.HfxError) as e:
        hfx.hfx_create(inv.lattice, inv.pos_frac, inv.rmt, inv.lmax, inv.Lmax, inv.P, inv.mesh, opt)
    assert e.value.code in (hfx.HFX_EDEVICE, hfx.HFX_EUNSUPPORTED)


def test_inversion_generator_obeys_its_stated_relations():
    """The generator's inversion variant, checked against the relation the
    library enforces (real c; A of the partner from A of the atom)."""
    s = S.make_system(4, mesh=(1, 2, 2), nb=4, no=2, aux=("count", 50, 50), inversion=True)
    p = S.inversion_partners(s.pos_frac, s.rmt)
    for ik in range(s.n_k):
        assert not np.any(s.c[ik].imag)
        kf = s.kpoint_frac(ik)
        for a in range(s.n_atoms):
            b = int(p[a])
            ph = np.exp(2j * np.pi * kf @ np.round(s.pos_frac[a] + s.pos_frac[b]))
            for l in range(s.lmax + 1):
                for m in range(-l, l + 1):
                    for q in range(2):
                        x = s.A[ik][:, a, 2 * (l * l + l + m) + q]
                        y = s.A[ik][:, b, 2 * (l * l + l - m) + q]
                        assert np.abs(y - (-1) ** (l + m) * ph * np.conj(x)).max() < 1e-14
    assert np.array_equal(s.R[0], s.R[p[0]]) and np.array_equal(s.mu[0], s.mu[p[0]])
