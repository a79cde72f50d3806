"""Batched discovery (traversal launches over many uneven scenes, replayed
from a CUDA graph) gives, scene by scene, exactly the path set of the
per-scene plain trace, before and after a frame update; and, on a strided
ray subset, the oracle's path set and fields scene by scene."""
import numpy as np
import pytest

import oracle
from helpers import compare_accepted, compare_field, rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small_batch(n=10, seed=3):
    """Uneven scenes shaped like the 64-scene batch, at reduced ray counts."""
    out = []
    for s in S.batched_scenes(seed=seed, n=n):
        s.n_rays = int(min(s.n_rays, 400_000))
        out.append(s)
    return out


def test_batched_equals_sequential(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("EMRT_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2303_10521_gb300 import engine
    descs = _small_batch()
    scs = []
    for d in descs:
        g = engine.Scene(d)
        g.update(d.frame(0))
        scs.append(g)
    caps = [max(4096, 8 * g.n_tx * g.n_rx) for g in scs]
    b = engine.Batch(scs, capacity=caps, autotune=True)
    assert (tmp_path / "tune.json").exists()
    for frame in (0, 2):
        if frame:
            for d, g in zip(descs, scs):
                g.update(d.frame(frame))
        for rep in range(2):  # first call captures the graph, second replays it
            b.trace_async()
            st = b.sync()
            assert st["error_bits"] == 0
            for d, g, o in zip(descs, scs, b.outs):
                ref = g.trace(capacity=o.capacity).records()
                got = o.records()
                assert got.shape == ref.shape, (d.name, got.shape, ref.shape)
                assert np.array_equal(got, ref), d.name
    assert "block" in b.config()


@pytest.mark.parametrize("breadth_first", [False, True])
def test_batch_forms_equal_sequential(breadth_first):
    """Untuned batches of either traversal form (depth-first: one launch for
    all bounces; breadth-first: one launch per bounce with the ray sort)
    give the per-scene traces' records, and say which form they run."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    descs = _small_batch(n=6, seed=11)
    scs = []
    for d in descs:
        g = engine.Scene(d)
        g.update(d.frame(0))
        scs.append(g)
    caps = [max(4096, 8 * g.n_tx * g.n_rx) for g in scs]
    b = engine.Batch(scs, capacity=caps, breadth_first=breadth_first)
    assert ("depth_first" in b.config()) != breadth_first, b.config()
    b.trace_async()
    assert b.sync()["error_bits"] == 0
    for d, g, o in zip(descs, scs, b.outs):
        ref = g.trace(capacity=o.capacity).records()
        assert np.array_equal(o.records(), ref), d.name


def test_trace_batched_one_call():
    """emrt_trace_batched: the first call captures, later calls replay, the
    outputs equal the per-scene traces; destroying a scene drops its batch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    descs = _small_batch(n=5, seed=7)
    scs = []
    for d in descs:
        g = engine.Scene(d)
        g.update(d.frame(0))
        scs.append(g)
    caps = [max(4096, 8 * g.n_tx * g.n_rx) for g in scs]
    refs = [g.trace(capacity=c).records() for g, c in zip(scs, caps)]
    outs = [engine.Paths(c, scs[0].device) for c in caps]
    for _ in range(3):
        engine.trace_batched(scs, outs)
        for o, r in zip(outs, refs):
            assert np.array_equal(o.records(), r)
    # after a frame update the replay traces the new poses
    for d, g in zip(descs, scs):
        g.update(d.frame(1))
    refs1 = [g.trace(capacity=c).records() for g, c in zip(scs, caps)]
    engine.trace_batched(scs, outs)
    for o, r in zip(outs, refs1):
        assert np.array_equal(o.records(), r)
    del scs[2]   # destroys that scene and with it the registered batch
    import gc
    gc.collect()
    engine.trace_batched(scs, [outs[i] for i in (0, 1, 3, 4)])
    for o, r in zip([outs[i] for i in (0, 1, 3, 4)], [refs1[i] for i in (0, 1, 3, 4)]):
        assert np.array_equal(o.records(), r)


@pytest.mark.parametrize("breadth_first", [False, True])
def test_batched_oracle_parity(breadth_first):
    """The batched form against the oracle, not only against the per-scene
    GPU traces: a 10-scene batch of uneven scenes traced together on a
    strided subset of each scene's rays (about 4000 per transmitter), then,
    for four of its scenes -- 18 vehicles and K = 4; 423 vehicles and K = 2;
    no vehicles and K = 4; 15k faces, 58 vehicles, K = 4 -- the accepted
    path set equals the oracle's on the same rays except flagged paths, and
    the field of every accepted path matches the oracle's FP64 field."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    descs = S.batched_scenes(seed=3, n=10)
    scs, params = [], []
    for i, d in enumerate(descs):
        g = engine.Scene(d)
        g.update(d.frame(0))
        scs.append(g)
        stride = max(1, d.n_rays // 4000)
        params.append(dict(stride=stride, offset=i % stride))
    caps = [max(4096, 8 * g.n_tx * g.n_rx) for g in scs]
    b = engine.Batch(scs, params=params, capacity=caps, breadth_first=breadth_first)
    b.trace_async()
    assert b.sync()["error_bits"] == 0
    checked, with_paths = 0, 0
    for i in (1, 4, 6, 8):
        d, g, out, p = descs[i], scs[i], b.outs[i], params[i]
        o = oracle.OracleScene(d, d.frame(0))
        cands, ray_marg, _ = oracle.trace(o, d.n_rays, d.max_depth, offset=p["offset"],
                                          stride=p["stride"])
        ga = rec_to_paths(out.records())
        rc = compare_accepted(o, ga, cands, ray_marg)
        assert not rc["missing"] and not rc["extra_bad"], (d.name, rc)
        with_paths += rc["n_gpu"] > 0
        ch = g.channel(out, d.freqs[0])
        po = ch.path[:out.n()].cpu().numpy()
        rf = compare_field(po[:, 0] + 1j * po[:, 1], po[:, 2], po[:, 3],
                           *oracle.field(o, ga, d.freqs[0]))
        assert rf["ok"], (d.name, rf)
        checked += rc["n_gpu"]
    assert checked > 50 and with_paths >= 3, (checked, with_paths)


def test_batch_trace_inside_a_caller_graph():
    """After its first call, emrt_batch_trace on a stream the caller captures
    is recorded into the caller's CUDA graph: replaying that graph after a
    frame update gives the per-scene traces' records of the new poses."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    descs = _small_batch(n=4, seed=5)
    scs = []
    for d in descs:
        g = engine.Scene(d)
        g.update(d.frame(0))
        scs.append(g)
    caps = [max(4096, 8 * g.n_tx * g.n_rx) for g in scs]
    b = engine.Batch(scs, capacity=caps)
    b.trace_async()
    b.sync()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, capture_error_mode="thread_local"):
        b.trace_async(stream=torch.cuda.current_stream())
    for frame in (1, 2):
        for d, g in zip(descs, scs):
            g.update(d.frame(frame))
        torch.cuda.synchronize()
        gr.replay()
        torch.cuda.synchronize()
        assert b.sync()["error_bits"] == 0
        for d, g, o in zip(descs, scs, b.outs):
            ref = g.trace(capacity=o.capacity).records()
            assert np.array_equal(o.records(), ref), (frame, d.name)
