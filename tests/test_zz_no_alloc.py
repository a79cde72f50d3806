"""The allocation-free adjoint entry point, emrt_channel_backward_noalloc.

Some callers cannot call cudaMalloc once they are running: applications whose
device memory belongs to another allocator or is capped, and real-time loops
that allocate everything up front so that no call stalls in the allocator.  For them the library
offers this variant of emrt_channel_backward, whose scratch is a fixed device
array inside libemrt.so.  This test calls it through the C-ABI, twice in a
row, and checks both results against the existing entry point; it also checks
that sizes beyond the array's capacity are refused.  It lives in its own file,
collected last, and passes alone or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grads(lib, fn, g, paths, mats, freq, cot, name):
    from paper_2303_10521_gb300 import _native as N
    d = g.device
    ge = torch.full((int(mats.n_mat),), float("nan"), dtype=torch.float64, device=d)
    gs = torch.full_like(ge, float("nan"))
    gt = torch.full((g.n_tx, 3), float("nan"), dtype=torch.float64, device=d)
    pc = paths.c()
    code = fn(g.h, C.byref(pc), C.byref(mats), float(freq), C.c_void_p(cot.data_ptr()),
              C.c_void_p(ge.data_ptr()), C.c_void_p(gs.data_ptr()), C.c_void_p(gt.data_ptr()),
              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(code, name)
    torch.cuda.synchronize()
    return ge.cpu().numpy(), gs.cpu().numpy(), gt.cpu().numpy()


def test_noalloc_adjoint_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import _native as N, engine
    lib = N.load()
    sc = S.district_scene(seed=4)
    g = engine.Scene(sc)
    g.update(sc.frame(0))
    paths = g.trace(stride=7)
    assert 0 < paths.n() <= paths.capacity <= N.NOALLOC_MAX_PATHS
    freq = sc.freqs[0]
    rng = np.random.default_rng(11)
    cot = torch.as_tensor(rng.normal(size=(g.n_tx, g.n_rx, 2)), device=g.device)
    mats = g._mat()
    ref = _grads(lib, lib.emrt_channel_backward, g, paths, mats, freq, cot,
                 "emrt_channel_backward")
    assert all(np.isfinite(r).all() for r in ref)
    for call in range(2):  # the shared array keeps the previous call's contents
        got = _grads(lib, lib.emrt_channel_backward_noalloc, g, paths, mats, freq, cot,
                     "emrt_channel_backward_noalloc")
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0.0)

    # a path buffer larger than the fixed array is refused before any launch
    big = engine.Paths(N.NOALLOC_MAX_PATHS + 1, g.device)
    with pytest.raises(N.EmrtError) as ei:
        _grads(lib, lib.emrt_channel_backward_noalloc, g, big, mats, freq, cot,
               "emrt_channel_backward_noalloc")
    assert ei.value.code == 1

    # NaN materials: reported at the next sync like the allocating adjoint
    nan_eps = torch.full_like(g.eps_r, float("nan"))  # kept alive across the call
    nan = g._mat(eps_r=nan_eps)
    _grads(lib, lib.emrt_channel_backward_noalloc, g, paths, nan, freq, cot,
           "emrt_channel_backward_noalloc")
    with pytest.raises(N.EmrtError) as ei:
        g.sync()
    assert ei.value.code == 7
    g.sync()
