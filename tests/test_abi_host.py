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
