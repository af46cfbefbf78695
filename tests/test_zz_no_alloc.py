"""The allocation-free q->0 bracket entry point (hfx_q0_bracket_noalloc).

Callers whose device memory is owned by another allocator, or that must not
trigger the synchronisation of cudaMalloc/cudaFree, use this variant: its
scratch is a fixed array inside the library.  The test calls it twice in a
row through the C ABI and compares each result with the context-based entry
point hfx_get_q0_bracket (same kernels and summation order, so the results
agree to the last bits).  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1003_0524_gb300 import hfx
from paper_1003_0524_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1003_0524_gb300 import build
    build.build()
    hfx.load()
    return torch


@pytest.mark.parametrize("cfg,mesh", [(1, (4, 4, 4)), (0, (2, 2, 2))])
def test_noalloc_bracket_matches_context_entry_point(torch_cuda, cfg, mesh):
    torch = torch_cuda
    s = S.make_system(cfg, mesh=mesh, nb=2, no=1)
    with hfx.Context(s, precision="fp64") as c:
        ref = c.q0_bracket()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for i in range(2):  # two calls in a row share the library's scratch array
        hfx.hfx_q0_bracket_noalloc(s.lattice, s.mesh, 0.005, out.data_ptr() + 8 * i, stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert got[0] == pytest.approx(ref, rel=1e-13, abs=0)
    assert got[1] == pytest.approx(ref, rel=1e-13, abs=0)


def test_noalloc_rejects_oversized_and_bad_input(torch_cuda):
    torch = torch_cuda
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = np.eye(3) * 60.0  # large cell: the G box per k exceeds the fixed array
    with pytest.raises(hfx.HfxError) as e:
        hfx.hfx_q0_bracket_noalloc(big, (64, 64, 64), 0.005, out.data_ptr())
    assert e.value.code == hfx.HFX_EUNSUPPORTED
    with pytest.raises(hfx.HfxError) as e:
        hfx.hfx_q0_bracket_noalloc(np.eye(3) * 8.0, (0, 2, 2), 0.005, out.data_ptr())
    assert e.value.code == hfx.HFX_EINVAL
