"""The C-ABI library builds, loads and exports every entry point declared in
include/emrt.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "emrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(emrt_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    from paper_2303_10521_gb300 import build, _native
    build.build()
    lib = ctypes.CDLL(_native.LIB_PATH)
    names = _declared()
    assert "emrt_trace" in names and "emrt_channel" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.SIGNATURES)


def test_status_strings_without_gpu():
    from paper_2303_10521_gb300 import _native
    lib = _native.load()
    assert lib.emrt_status_string(4) == b"buffer capacity exceeded"
    assert lib.emrt_status_string(0) == b"ok"


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2303_10521_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "emrt_oracle" not in txt, f


def test_paths_checkpoint_roundtrip(tmp_path):
    """A path set saved and loaded again (checkpoint/resume of a cache) keeps
    its records and count; the capacity can grow on load."""
    import torch
    from paper_2303_10521_gb300 import engine
    p = engine.Paths(16, "cpu")
    recs = np.arange(5 * 8, dtype=np.uint32).reshape(5, 8) * np.uint32(2654435761)
    p.rec[:5] = torch.from_numpy(recs.view(np.int32))
    p.count.fill_(5)
    f = str(tmp_path / "cache.npy")
    p.save(f)
    q = engine.Paths.load(f, "cpu", capacity=64)
    assert q.capacity == 64 and q.n() == 5
    assert np.array_equal(q.records(), recs)
    e = engine.Paths(4, "cpu")
    e.save(f)
    assert engine.Paths.load(f, "cpu").n() == 0


def test_heatmap_export(tmp_path):
    """Per-receiver dBm heat-map arrays: 1 W is 30 dBm, 1 mW 0 dBm, no path
    -inf; with positions the file holds (x, y, z, dBm) rows."""
    import torch
    from paper_2303_10521_gb300 import engine
    rx = torch.tensor([[1.0, 2.0], [1e-3, 0.5], [0.0, 0.0]], dtype=torch.float64)
    ch = engine.ChannelResult(torch.zeros(1, 4, dtype=torch.float64),
                              torch.zeros(1, 3, 8, dtype=torch.float64), rx)
    d = engine.rx_dbm(ch)
    assert d[0] == 30.0 and abs(d[1]) < 1e-12 and d[2] == -np.inf
    assert abs(engine.rx_dbm(ch, coherent=False)[0] - (30.0 + 10 * np.log10(2.0))) < 1e-12
    pos = np.array([[0, 0, 1.5], [10, 0, 1.5], [0, 20, 1.6]])
    f = str(tmp_path / "heat.npy")
    engine.save_heatmap(f, ch, rx_pos=pos)
    h = np.load(f)
    assert h.shape == (3, 4) and np.array_equal(h[:, :3], pos) and h[0, 3] == 30.0
    engine.save_heatmap(f, ch)
    assert np.load(f).shape == (3,)
