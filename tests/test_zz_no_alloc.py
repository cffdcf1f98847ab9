"""mm_emulated_noalloc: the emulated product for callers that cannot allocate a
device workspace (its scratch lives in the library's fixed 64 MiB device array).

Called through the C ABI, twice in a row on different inputs -- the second with
smaller magnitudes and a different shape, so any scratch state left by the first
call (stale column maxima, stale slices) would change the result -- and each
output is compared with mm_emulated's on the same inputs, bit for bit (the
tolerance every emulated-product test here uses)."""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1106_1347_gb300 import _native, build

    build.build()
    return _native


def _with_workspace(lib, ta, tb, s):
    import torch

    n, p = ta.shape
    m = tb.shape[1]
    c = torch.empty((n, m), dtype=torch.float64, device="cuda")
    need = lib.mm_emulated_workspace_bytes(n, p, m, 0, s, 1e-14)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mm_emulated(n, p, m, ctypes.c_void_p(ta.data_ptr()), p, ctypes.c_void_p(tb.data_ptr()), m,
                         ctypes.c_void_p(c.data_ptr()), m, 0, s, 1e-14, ctypes.c_void_p(ws.data_ptr()), need, st)
    assert rc == 0, lib.mm_last_error()
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _no_alloc(lib, ta, tb, s):
    import torch

    n, p = ta.shape
    m = tb.shape[1]
    c = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mm_emulated_noalloc(n, p, m, ctypes.c_void_p(ta.data_ptr()), p, ctypes.c_void_p(tb.data_ptr()), m,
                                 ctypes.c_void_p(c.data_ptr()), m, 0, s, 1e-14, st)
    assert rc == 0, lib.mm_last_error()
    torch.cuda.synchronize()
    return c.cpu().numpy()


def test_no_alloc_matches_workspace_version_twice(native):
    import torch

    lib = native.lib()
    assert lib.mm_emulated_noalloc_capacity() == 64 << 20
    calls = [
        (S.loguniform(300, 700, S.stream_seed(5, 0)), S.loguniform(700, 260, S.stream_seed(5, 1)), 8),
        (S.uniform(190, 450, S.stream_seed(5, 2)) * 1e-3, S.uniform(450, 333, S.stream_seed(5, 3)) * 1e-3, 8),
    ]
    for a, b, s in calls:
        ta = torch.from_numpy(a).cuda()
        tb = torch.from_numpy(b).cuda()
        want = _with_workspace(lib, ta, tb, s)
        got = _no_alloc(lib, ta, tb, s)
        assert np.array_equal(got, want)


def test_no_alloc_rejects_oversize(native):
    import torch

    lib = native.lib()
    need = lib.mm_emulated_workspace_bytes(2048, 2048, 2048, 0, 8, 1e-14)
    assert need > lib.mm_emulated_noalloc_capacity()
    a = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    c = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mm_emulated_noalloc(2048, 2048, 2048, ctypes.c_void_p(a.data_ptr()), 2048, ctypes.c_void_p(a.data_ptr()),
                                 2048, ctypes.c_void_p(c.data_ptr()), 2048, 0, 8, 1e-14, st)
    assert rc == -3  # MM_ERR_NOMEM
    assert b"static" in lib.mm_last_error()
