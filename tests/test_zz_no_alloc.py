"""dvnr_error_stats_noalloc: the FP64 error statistics for callers that must
not allocate device memory when they ask for the error (an in situ pipeline
whose simulation keeps the device memory for itself, or a time step that
cannot afford the implicit device synchronisation of cudaMalloc/cudaFree).

The call keeps its scratch in a fixed array inside the library; here it is
checked against dvnr_error_stats (which allocates its scratch) on two calls
in a row, with the tolerance of the error-statistics test, and its size limit
is checked. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import _abi as A

    return A


def _stats(A, name, a, b):
    out = (C.c_double * 2)()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A.call(name, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), a.numel(),
           C.cast(out, C.c_void_p), stream)
    return out[0], out[1]


def test_noalloc_error_stats_matches_allocating_call(lib):
    rng = np.random.default_rng(11)
    # two calls in a row with different sizes: the second must not see the
    # first call's partial sums left in the shared scratch
    for n, scale in ((3_000_017, 1e-3), (150_001, 0.25)):
        a = rng.normal(size=n).astype(np.float32)
        b = (a + rng.normal(scale=scale, size=n)).astype(np.float32)
        ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        want = _stats(lib, "dvnr_error_stats", ta, tb)
        got = _stats(lib, "dvnr_error_stats_noalloc", ta, tb)
        assert got[0] == pytest.approx(want[0], rel=1e-12)
        assert got[1] == want[1]
        d = a.astype(np.float64) - b.astype(np.float64)
        assert got[0] == pytest.approx(float((d * d).sum()), rel=1e-12)


def test_noalloc_error_stats_limits(lib):
    t = torch.zeros(4, device="cuda")
    assert _stats(lib, "dvnr_error_stats_noalloc", t[:0], t[:0]) == (0.0, 0.0)
    out = (C.c_double * 2)()
    rc = lib.load().dvnr_error_stats_noalloc(C.c_void_p(t.data_ptr()), C.c_void_p(t.data_ptr()),
                                             (1 << 28) + 1, C.cast(out, C.c_void_p), None)
    assert rc == 1  # DVNR_E_INVALID: beyond the scratch maximum, rejected before any work
    assert b"exceeds" in lib.load().dvnr_last_error()
