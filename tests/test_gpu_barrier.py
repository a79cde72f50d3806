"""The bounded grid barrier of the per-frame cooperative tree builds: it
completes when every block arrives, and when an arrival never comes (a block
count that nothing can reach) every block gives up after the poll limit,
reports it, and the context stays usable."""
import ctypes as C
import time

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import _native
    return _native.load()


def _run(lib, missing):
    passed, timed = C.c_uint32(99), C.c_uint32(99)
    rc = lib.emrt_selftest_grid_barrier(missing, C.byref(passed), C.byref(timed))
    return rc, passed.value, timed.value


def test_barrier_completes(lib):
    assert _run(lib, 0) == (0, 4, 0)


def test_barrier_gives_up_and_context_survives(lib):
    t0 = time.perf_counter()
    rc, passed, timed = _run(lib, 1)
    dt = time.perf_counter() - t0
    assert rc == 0 and passed == 0 and timed == 1
    assert dt < 5.0
    assert _run(lib, 0) == (0, 4, 0)  # the next launch works
    x = torch.arange(8, device="cuda").sum().item()
    assert x == 28


def test_invalid_arguments(lib):
    passed = C.c_uint32()
    assert lib.emrt_selftest_grid_barrier(0, C.byref(passed), None) == 1
    assert lib.emrt_selftest_grid_barrier(2000, C.byref(passed), C.byref(passed)) == 1
