"""Static-hit cache (EMRT_TRACE_STATIC_CACHE): the output must be the plain
trace's output bit for bit -- same unique candidates with the same flags and
ray indices, same segment and candidate counts -- on a cold cache, on later
frames with moved vehicles and receivers, after a transmitter moved and
after the reflection depth grew."""
import dataclasses

import numpy as np
import pytest

from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine as E
    return E


def _both(g, **kw):
    a = g.trace(keep_rejected=True, **kw).records()
    sa = dict(g.last_stats)
    b = g.trace(keep_rejected=True, static_cache=True, **kw).records()
    sb = dict(g.last_stats)
    return a, sa, b, sb


def _same(a, sa, b, sb):
    assert np.array_equal(a, b)
    assert sa["segments"] == sb["segments"]
    assert sa["candidates"] == sb["candidates"]
    assert sa["accepted"] == sb["accepted"]


@pytest.mark.parametrize("seed,stride", [(0, 7), (4, 3)])
def test_district_frames_identical(engine, seed, stride):
    sc = S.district_scene(seed=seed)
    g = engine.Scene(sc)
    reuse = []
    for k in (0, 1, 2, 5, 9, 30):
        g.update(sc.frame(k))
        a, sa, b, sb = _both(g, stride=stride)
        _same(a, sa, b, sb)
        reuse.append(sb["static_reused"] / sum(sb["segments"]))
    assert reuse[0] == 0.0          # cold cache: everything traced and stored
    assert min(reuse[1:]) > 0.8, reuse


def test_transmitter_move_and_depth_change(engine):
    sc = S.district_scene(seed=5)
    g = engine.Scene(sc)
    fr = sc.frame(0)
    g.update(fr)
    _same(*_both(g, stride=5))
    _same(*_both(g, stride=5))
    moved = dataclasses.replace(fr, tx_pos=fr.tx_pos + np.float32([[0.5, 0.0, 0.0],
                                                                   [0.0, 0.0, 0.0]]))
    g.update(moved)
    a, sa, b, sb = _both(g, stride=5)
    _same(a, sa, b, sb)
    # only the transmitter that did not move reuses its chains
    assert 0 < sb["static_reused"] < 0.75 * sum(sb["segments"])
    _same(*_both(g, stride=5))
    # one more reflection than the cache was built for: it is rebuilt
    a, sa, b, sb = _both(g, stride=5, max_depth=sc.max_depth + 1)
    _same(a, sa, b, sb)
    assert sb["static_reused"] == 0
    _same(*_both(g, stride=5, max_depth=sc.max_depth + 1))
    # a smaller depth reuses the deeper cache
    a, sa, b, sb = _both(g, stride=5, max_depth=sc.max_depth - 1)
    _same(a, sa, b, sb)
    assert sb["static_reused"] > 0


def test_toy_and_single_leaf_scenes(engine):
    sc = S.toy_scene(seed=3)
    g = engine.Scene(sc)
    g.update(sc.frame(0))
    for _ in range(2):
        _same(*_both(g))
    # one wall only (a single-leaf static BVH), no vehicles
    wall = S.rect_wall_x(20.0, -50, 50, 0, 30, facing=-1)
    sc2 = S.custom_scene([wall], [S.MAT_CONCRETE], (0, 0, 5), [(3.0, 10.0, 2.0), (5, -9, 1)])
    g2 = engine.Scene(sc2)
    g2.update(sc2.frame(0))
    for _ in range(2):
        _same(*_both(g2, n_rays=50_000, max_depth=2))
