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
