"""The allocation-free forward entry point, psr_p2p_forces_noalloc.

Some callers cannot allocate device memory (a framework that owns all device
memory through its own pool, a context where an allocation may block, a
policy of no allocations after start-up).  psr_p2p_forces_noalloc serves them:
its scratch is a fixed array inside the library.  These tests call it through
the C ABI and check it against psr_p2p_forces on the same uploaded leaf set,
twice in a row (the array keeps the previous call's contents).  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
psr = pytest.importorskip("paper_2107_14008_gb300")
from paper_2107_14008_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14008_gb300 import build
    build.build()


def _clustered(n=6000, L=60.0, seed=3):
    rng = np.random.default_rng(seed)
    pos, _ = synth.nfw_clustered(n, L, 0.6, 6, rng)
    r_s, r_c = synth.box_params(L, 16)
    return pos, rng.uniform(0.2, 2.0, n), L, r_s, r_c


@pytest.mark.parametrize("kw", [
    dict(precision=psr.PSR_FP32_TABLE, table_n=1024, interp=psr.PSR_LINEAR),
    dict(precision=psr.PSR_FP32_TABLE, table_n=4096, interp=psr.PSR_CUBIC),
    dict(precision=psr.PSR_FP32_TABLE, kernel=psr.PSR_KERNEL_PACKED),
    dict(precision=psr.PSR_FP32_EXACT),
    dict(precision=psr.PSR_FP64),
])
def test_noalloc_matches_allocating_entry_point(kw):
    """Both entry points launch the same kernel on the same inputs, and each
    target's sum runs in a fixed order, so the results must be equal bit for
    bit: a table rebuilt wrongly or counters left over from the previous call
    would show."""
    pos, mass, L, r_s, r_c = _clustered()
    lv = psr.Leaves.build(pos, mass, L, r_s, r_c).upload()
    opts = psr.Options(**kw)
    ref = lv.forces(opts).clone()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the second call starts from the first call's array contents
        out = torch.full_like(ref, float("nan"))
        capi.psr_p2p_forces_noalloc(lv._h, opts.c(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_a_table_beyond_its_array():
    pos, mass, L, r_s, r_c = _clustered(n=500)
    lv = psr.Leaves.build(pos, mass, L, r_s, r_c).upload()
    out = torch.empty((500, 3), dtype=torch.float32, device="cuda")
    opts = psr.Options(precision=psr.PSR_FP32_TABLE, table_n=8192)
    with pytest.raises(capi.PsrError) as e:
        capi.psr_p2p_forces_noalloc(lv._h, opts.c(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.code == capi.PSR_E_ARG
    assert "4096" in str(e.value)
