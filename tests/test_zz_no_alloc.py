"""The allocation-free window sieve, mertens_sieve_M_noalloc (GPU).

Some callers cannot allocate device memory at the point where they need
M(y): a framework that has reserved the device memory for its own pool, or a
latency-critical loop that cannot afford cudaMalloc/cudaFree (which
synchronise the device and may fail).  For them the library keeps a fixed
scratch array on the device.  This file checks, through the C ABI, that the
allocation-free call returns exactly what the allocating mertens_sieve_M
returns, on two calls in a row that reuse that scratch, and that windows
beyond its stated limit are refused.  It is collected last on purpose.
"""
import numpy as np
import pytest

import paper_1108_0135_gb300 as pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.load()
    yield


def allocating(y1, length, carry):
    out = torch.empty(length, dtype=torch.int32, device="cuda")
    pm.mertens_sieve_M(y1, length, carry, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_equals_allocating_entry_point_on_consecutive_calls():
    # two calls in a row with different windows: the second reuses (and must
    # fully overwrite) the scratch the first one left behind
    # the last window ends just below the stated limit y < 2^40, where the
    # allocating call takes the byte sieve and this one the 16-bit sieve
    for y1, length, carry in [(10**9 + 7, 300_011, 123_456), (1, 1 << 21, 0),
                              ((1 << 40) - (1 << 21), 1 << 21, 0)]:
        out = torch.full((length,), -7, dtype=torch.int32, device="cuda")
        pm.mertens_sieve_M_noalloc(y1, length, carry, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, allocating(y1, length, carry)), (y1, length)


def test_noalloc_refuses_windows_beyond_its_limit():
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    for y1, length in [(1, (1 << 21) + 1), (1 << 40, 1), ((1 << 40) - 8, 16)]:
        with pytest.raises(pm.MertensError) as ei:
            pm.mertens_sieve_M_noalloc(y1, length, 0, out)
        assert ei.value.code == pm.MERTENS_EINVAL
