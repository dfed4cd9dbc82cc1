"""igg_reduce_noalloc, the reduction that allocates nothing in the library,
called through the C ABI and checked against igg_reduce on two calls in a
row. It serves callers that cannot allocate device memory while they reduce
(a fixed device-memory budget, an allocator that owns all memory, capture
regions that forbid allocation calls)."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

OPS = (0, 1, 2, 3)  # MAX, SUM, SUM_DIV, SUM_SQDIFF


@pytest.fixture(scope="module")
def L():
    from paper_2211_15716_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2211_15716_gb300 import igg
    lib = igg.lib()
    lib.igg_reduce_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.igg_reduce_noalloc.restype = ctypes.c_int
    return lib


def _noalloc(L, op, a, b, code):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.igg_reduce_noalloc(op, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(),
                              code, ctypes.c_void_p(out.data_ptr()), s)
    assert rc == 0, L.igg_last_error().decode()
    return out.item()


@pytest.mark.parametrize("dtype,code", [(torch.float64, 0), (torch.float32, 1), (torch.bfloat16, 2)])
def test_noalloc_matches_reduce_two_calls(L, dtype, code):
    from paper_2211_15716_gb300 import igg
    rng = np.random.default_rng(5)
    n = 3 * 65536 + 12345  # several chunks and a ragged last one
    a = torch.from_numpy(rng.uniform(1.0, 3.0, n)).to(dtype).cuda()
    b = torch.from_numpy(rng.uniform(0.4, 0.7, n)).to(dtype).cuda()
    for op in OPS:
        ref = igg.reduce(op, a, b).item()
        for _ in range(2):
            got = _noalloc(L, op, a, b, code)
            if op == 0:
                assert got == ref
            else:
                assert got == pytest.approx(ref, rel=1e-13)


def test_noalloc_smaller_call_after_larger(L):
    """A small call right after a large one gives the small input's result
    (stale partial sums from the larger call are never read)."""
    from paper_2211_15716_gb300 import igg
    big = torch.ones(10 * 65536, dtype=torch.float64, device="cuda")
    small = torch.full((1000,), 2.0, dtype=torch.float64, device="cuda")
    assert _noalloc(L, 1, big, big, 0) == 10 * 65536
    assert _noalloc(L, 1, small, small, 0) == 2000.0
    assert _noalloc(L, 1, small, small, 0) == igg.reduce(1, small).item()


def test_noalloc_rejects_too_large(L):
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = L.igg_reduce_noalloc(1, ctypes.c_void_p(buf.data_ptr()), None, 32768 * 65536 + 1, 0,
                              ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert "exceeds the maximum" in L.igg_last_error().decode()


def _call(L, fn, op, a, b, n, code):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    pa = ctypes.c_void_p(a.data_ptr()) if a is not None else None
    pb = ctypes.c_void_p(b.data_ptr()) if b is not None else None
    rc = getattr(L, fn)(op, pa, pb, n, code, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0, L.igg_last_error().decode()
    torch.cuda.synchronize()
    return out.item()


def test_noalloc_empty_input_gives_identity(L):
    """n == 0 (no input pointers needed): SUM gives 0 and MAX gives -inf,
    the same as igg_reduce."""
    from paper_2211_15716_gb300 import igg
    L.igg_reduce.argtypes = L.igg_reduce_noalloc.argtypes
    for fn in ("igg_reduce_noalloc", "igg_reduce"):
        assert _call(L, fn, 1, None, None, 0, 0) == 0.0
        assert _call(L, fn, 0, None, None, 0, 0) == float("-inf")
    assert igg.reduce(1, torch.empty(0, dtype=torch.float64, device="cuda")).item() == 0.0


def test_noalloc_sum_and_max_without_b(L):
    """SUM and MAX read only a: b may be NULL, with the results of igg_reduce."""
    from paper_2211_15716_gb300 import igg
    rng = np.random.default_rng(6)
    a = torch.from_numpy(rng.uniform(-2.0, 3.0, 2 * 65536 + 7)).cuda()
    assert _call(L, "igg_reduce_noalloc", 0, a, None, a.numel(), 0) == igg.reduce(0, a).item()
    assert _call(L, "igg_reduce_noalloc", 1, a, None, a.numel(), 0) == pytest.approx(
        igg.reduce(1, a).item(), rel=1e-13)
    assert _call(L, "igg_reduce_noalloc", 1, a, None, a.numel(), 0) == pytest.approx(
        float(a.sum()), rel=1e-12)
