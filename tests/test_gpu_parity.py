"""GPU parity: the CUDA path through the C-ABI against the CPU oracle on the
same seeded inputs (element by element), plus closed forms."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from helpers import (compare_acceptance, compare_candidates, compare_field, rec_to_paths,
                     C_LIGHT)
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine as E
    return E


def _gpu(E, sc, frame=None, **kw):
    g = E.Scene(sc, **kw)
    g.update(frame if frame is not None else sc.frame(0))
    return g


def _field(g, paths, freq, **kw):
    ch = g.channel(paths, freq, **kw)
    n = paths.n()
    po = ch.path[:n].cpu().numpy()
    return po[:, 0] + 1j * po[:, 1], po[:, 2], po[:, 3], ch


# ---------------------------------------------------------------------------
def test_friis_two_ray_single_wall_closed_forms(engine):
    f = 3.5e9
    k = 2 * math.pi * f / C_LIGHT
    lam = C_LIGHT / f
    # free space
    sc = S.custom_scene([], [], (0, 0, 10), (250.0, 40.0, 1.5), freq=f)
    g = _gpu(engine, sc)
    p = g.trace(n_rays=200_000, max_depth=2)
    recs = rec_to_paths(p.records())
    assert len(recs) == 1 and recs["depth"][0] == 0
    a, tau, fd, _ = _field(g, p, f)
    d = float(np.linalg.norm(np.float32([250.0, 40.0, 1.5]).astype(float) - [0, 0, 10]))
    expect = lam / (4 * math.pi * d) * np.exp(-1j * k * d)
    assert abs(a[0] - expect) <= 1e-9 * abs(expect)
    # two-ray ground
    ground = S.rect_xy(-2e3, -2e3, 2e3, 2e3)
    sc = S.custom_scene([ground], [S.MAT_GROUND], (0, 0, 30), (300.0, 0.0, 1.5), freq=f)
    g = _gpu(engine, sc)
    p = g.trace(n_rays=400_000, max_depth=2)
    recs = rec_to_paths(p.records())
    assert sorted(recs["depth"].tolist()) == [0, 1]
    a, tau, fd, ch = _field(g, p, f)
    o = oracle.OracleScene(sc, sc.frame(0))
    a_o, tau_o, fd_o = oracle.field(o, recs, f)
    r = compare_field(a, tau, fd, a_o, tau_o, fd_o)
    assert r["ok"], r
    h = ch.pair[0, 0].cpu().numpy()
    assert complex(h[0], h[1]) == pytest.approx(complex(a_o.sum()), rel=1e-9)
    # single wall, s polarised
    wall = S.rect_wall_x(20.0, -100, 100, -50, 50, facing=-1)
    sc = S.custom_scene([wall], [S.MAT_CONCRETE], (0, 0, 5), (3.0, 40.0, 5.0), freq=28e9)
    g = _gpu(engine, sc)
    p = g.trace(n_rays=400_000, max_depth=1)
    recs = rec_to_paths(p.records())
    assert sorted(recs["depth"].tolist()) == [0, 1]
    a, tau, fd, _ = _field(g, p, 28e9)
    o = oracle.OracleScene(sc, sc.frame(0))
    r = compare_field(a, tau, fd, *oracle.field(o, recs, 28e9))
    assert r["ok"], r


def test_toy_scene_full_parity(engine):
    """Static toy scene, 100k rays, 2 reflections: discovery, acceptance,
    field and per-receiver reduction against the oracle."""
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    g = _gpu(engine, sc)
    o = oracle.OracleScene(sc, fr)
    allc = g.trace(keep_rejected=True)
    gu = rec_to_paths(allc.records())
    cands, ray_marg, _ = oracle.trace(o, sc.n_rays, sc.max_depth)
    rc = compare_candidates(gu, cands, ray_marg)
    assert not rc["missing"] and not rc["extra_bad"], rc
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra
    acc = g.trace()
    ga = rec_to_paths(acc.records())
    assert len(ga) == ra["n_acc_gpu"]
    # canonical order
    k = oracle.key_fields(ga)
    assert all(tuple(k[i]) < tuple(k[i + 1]) for i in range(len(k) - 1))
    a, tau, fd, ch = _field(g, acc, sc.freqs[0])
    a_o, tau_o, fd_o = oracle.field(o, ga, sc.freqs[0])
    rf = compare_field(a, tau, fd, a_o, tau_o, fd_o)
    assert rf["ok"], rf
    st = oracle.reduce(ga, a_o, tau_o, fd_o, 1, len(fr.rx_pos))
    pair = ch.pair.cpu().numpy()
    h_g = pair[..., 0] + 1j * pair[..., 1]
    h_o = st[..., 0] + 1j * st[..., 1]
    # per pair, the coherent sum may differ by the per-path tolerance summed
    sum_abs = np.zeros(h_o.shape)
    np.add.at(sum_abs, (ga["tx"].astype(int), ga["rx"].astype(int)), np.abs(a_o))
    assert np.all(np.abs(h_g - h_o) <= 1e-4 * sum_abs + 1e-30)
    assert pair[..., 7] == pytest.approx(st[..., 7])
    assert pair[..., 2] == pytest.approx(st[..., 2], rel=1e-6)
    assert pair[..., 3] == pytest.approx(st[..., 3], abs=1e-6)
    assert pair[..., 5] == pytest.approx(st[..., 5], rel=1e-9, abs=1e-15)
    coh, inc = oracle.rx_power(st, sc.tx_power_w)
    rx = ch.rx.cpu().numpy()
    assert rx[:, 0] == pytest.approx(coh, rel=1e-6)
    assert rx[:, 1] == pytest.approx(inc, rel=1e-6)


@pytest.mark.parametrize("stride,offset,form", [(97, 5, "depth_first"), (211, 0, "depth_first"),
                                                (131, 3, "wide_bvh")])
def test_district_subsample_parity(engine, stride, offset, form):
    """District (400 buildings, 200 vehicles, 1000 Rx, 2 Tx, K = 3) on a
    strided subset of the 1M rays, traced identically on both sides; the
    default depth-first discovery through the binary BVH and through the
    compressed 8-wide BVH."""
    sc = S.district_scene(seed=0)
    fr = sc.frame(0)
    g = _gpu(engine, sc)
    o = oracle.OracleScene(sc, fr)
    kw = dict(wide_bvh=True) if form == "wide_bvh" else {}
    allc = g.trace(stride=stride, offset=offset, keep_rejected=True, **kw)
    gu = rec_to_paths(allc.records())
    cands, ray_marg, _ = oracle.trace(o, sc.n_rays, sc.max_depth, offset=offset, stride=stride)
    rc = compare_candidates(gu, cands, ray_marg)
    assert not rc["missing"] and not rc["extra_bad"], {k: v for k, v in rc.items() if k != "bad"}
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra
    acc = g.trace(stride=stride, offset=offset, **kw)
    ga = rec_to_paths(acc.records())
    a, tau, fd, _ = _field(g, acc, 3.5e9)
    rf = compare_field(a, tau, fd, *oracle.field(o, ga, 3.5e9))
    assert rf["ok"], rf


def test_district_traversal_forms_identical(engine):
    """The depth-first chains (default), the breadth-first form with and
    without the ray sort, and both through the compressed 8-wide BVH,
    forward and backward: the same records bit for bit and the same segments
    per bounce."""
    sc = S.district_scene(seed=0)
    g = _gpu(engine, sc)
    forms = [dict(), dict(breadth_first=True), dict(breadth_first=True, sort_rays=False),
             dict(wide_bvh=True), dict(wide_bvh=True, breadth_first=True)]
    ref, ref_segs = None, None
    for kw in forms:
        rec = g.trace(stride=13, offset=7, keep_rejected=True, **kw).records()
        segs = g.last_stats["segments"]
        if ref is None:
            ref, ref_segs = rec, segs
            assert len(rec) > 100
        assert np.array_equal(rec, ref), kw
        assert segs == ref_segs, kw
    ids = torch.arange(0, g.n_rx, 7, dtype=torch.int32, device="cuda")
    b0 = g.trace_backward(ids, n_rays=20_000, keep_rejected=True).records()
    b1 = g.trace_backward(ids, n_rays=20_000, keep_rejected=True, breadth_first=True).records()
    b2 = g.trace_backward(ids, n_rays=20_000, keep_rejected=True, wide_bvh=True).records()
    assert len(b0) > 10 and np.array_equal(b0, b1) and np.array_equal(b0, b2)


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_scenes(engine, seed):
    """Property test on random tiny scenes (<= 25 static faces, 0-2 vehicles,
    K = 3): discovery equals the oracle's on the same rays except rays it
    flags, acceptance agrees except flagged paths, and the accepted set lies
    in the exhaustive image enumeration and holds >= 98 % of its power."""
    sc = S.tiny_scene(seed)
    fr = sc.frame(0)
    g = _gpu(engine, sc)
    o = oracle.OracleScene(sc, fr)
    gu = rec_to_paths(g.trace(keep_rejected=True).records())
    cands, ray_marg, _ = oracle.trace(o, sc.n_rays, sc.max_depth)
    rc = compare_candidates(gu, cands, ray_marg)
    assert not rc["missing"] and not rc["extra_bad"], rc
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra
    acc = rec_to_paths(g.trace().records())
    ex = oracle.enumerate_paths(o, sc.max_depth)
    kex = [tuple(r) for r in oracle.key_fields(ex).tolist()]
    kacc = {tuple(r) for r in oracle.key_fields(acc).tolist()}
    outside = [i for i, k in enumerate(oracle.key_fields(acc).tolist()) if tuple(k) not in set(kex)]
    if outside:  # only paths the oracle places within the margin
        _, vm = oracle.validate(o, acc[outside])
        assert (vm != 0).all(), acc[outside]
    a, _, _ = oracle.field(o, ex, sc.freqs[0])
    w = np.abs(a) ** 2
    assert sum(wi for k, wi in zip(kex, w) if k in kacc) >= 0.98 * w.sum()


def test_revalidate_cache_counts_evictions(engine):
    """emrt_revalidate_cache keeps what emrt_revalidate keeps and reports the
    number of records it removed."""
    sc = S.district_scene(seed=1)
    g = _gpu(engine, sc)
    p0 = g.trace(stride=53)
    p1 = g.trace(stride=53)
    n0 = p0.n()
    g.update(sc.frame(5))
    ev = g.revalidate_cache(p0)
    g.revalidate(p1)
    assert np.array_equal(p0.records(), p1.records())
    assert int(ev.item()) == n0 - p0.n() and int(ev.item()) > 0


def test_revalidation_and_merge(engine):
    """Cached frame: paths discovered at frame 0 revalidated with the poses of
    frame 3, flag by flag against the oracle; merge is a sorted union."""
    sc = S.district_scene(seed=1)
    g = _gpu(engine, sc)
    p0 = g.trace(stride=53)
    n0 = p0.n()
    assert n0 > 40
    fr3 = sc.frame(3)
    g.update(fr3)
    g.revalidate(p0, keep=True)
    recs = rec_to_paths(p0.records())
    assert len(recs) == n0
    o3 = oracle.OracleScene(sc, fr3)
    ra = compare_acceptance(o3, recs)
    assert ra["n_diff_unflagged"] == 0, ra
    g.revalidate(p0)
    kept = rec_to_paths(p0.records())
    assert len(kept) == int((recs["flag"] & 1).sum())
    assert oracle.key_fields(kept).tolist() == oracle.key_fields(recs[(recs["flag"] & 1) == 1]).tolist()
    fresh = g.trace(stride=53, offset=7)
    fk = rec_to_paths(fresh.records())
    cache = engine.Paths(len(kept) + len(fk) + 16, g.device)
    cache.rec[:len(kept)] = p0.rec[:len(kept)]
    cache.count.fill_(len(kept))
    g.merge(cache, fresh)
    merged = rec_to_paths(cache.records())
    want = sorted(set(map(tuple, oracle.key_fields(kept))) | set(map(tuple, oracle.key_fields(fk))))
    assert [tuple(r) for r in oracle.key_fields(merged)] == want
    # merging the union into itself changes nothing; an input out of
    # canonical order is reported at the next sync
    again = engine.Paths(cache.capacity, g.device)
    again.rec[:cache.n()] = cache.rec[:cache.n()]
    again.count.fill_(cache.n())
    g.merge(again, cache)
    g.sync()
    assert np.array_equal(again.records(), cache.records())
    bad = engine.Paths(cache.capacity, g.device)
    bad.rec[:len(kept)] = torch.flip(p0.rec[:len(kept)], dims=[0])
    bad.count.fill_(len(kept))
    g.merge(bad, fresh)
    from paper_2303_10521_gb300 import _native
    with pytest.raises(_native.EmrtError):
        g.sync()


@pytest.mark.parametrize("static_cache", [False, True])
def test_rediscover_equals_trace_and_merge(engine, static_cache):
    """Cached frames of the district: revalidation then rediscovery into the
    cache (candidates the cache holds are not validated again), and the
    rediscovery that revalidates on a side stream itself, give the records of
    revalidation, a separate trace and a merge, bit for bit."""
    sc = S.district_scene(seed=4)
    g = _gpu(engine, sc)
    first = g.trace(stride=29)
    a = engine.Paths(first.capacity * 4, g.device)
    b = engine.Paths(first.capacity * 4, g.device)
    c = engine.Paths(first.capacity * 4, g.device)
    for p in (a, b, c):
        p.rec[:first.n()] = first.rec[:first.n()]
        p.count.fill_(first.n())
    fresh = engine.Paths(first.capacity * 2, g.device)
    for k in (1, 2, 3):
        g.update(sc.frame(k))
        g.revalidate(a)
        g.trace_async(fresh, stride=97, offset=k, static_cache=static_cache)
        g.merge(a, fresh)
        st_a = g.sync()
        g.revalidate(b)
        g.rediscover(b, stride=97, offset=k, static_cache=static_cache)
        st_b = g.sync()
        assert st_b["accepted"] == b.n()
        assert st_a["segments"] == st_b["segments"]
        assert b.n() > first.n() // 2
        assert np.array_equal(a.records(), b.records()), k
        # the same with the revalidation inside the call (side stream)
        g.rediscover(c, stride=97, offset=k, static_cache=static_cache, revalidate=True)
        st_c = g.sync()
        assert st_c["error_bits"] == 0
        assert np.array_equal(a.records(), c.records()), k


def test_dynamic_frames_vehicle_paths(engine):
    """Several frames of the district: vehicle faces appear in paths, the
    vehicle BVH is refitted and rebuilt, and Doppler matches the oracle."""
    sc = S.district_scene(seed=2)
    g = engine.Scene(sc, rebuild_every=3)
    seen_vehicle = False
    for k in (0, 1, 2, 3, 4):
        fr = sc.frame(k)
        g.update(fr)
        p = g.trace(stride=101, offset=k)
        ga = rec_to_paths(p.records())
        o = oracle.OracleScene(sc, fr)
        ra = compare_acceptance(o, ga)
        assert ra["n_diff_unflagged"] == 0, ra
        a, tau, fd, _ = _field(g, p, 3.5e9)
        rf = compare_field(a, tau, fd, *oracle.field(o, ga, 3.5e9))
        assert rf["ok"], rf
        f = ga["face"]
        seen_vehicle |= bool(((f >= sc.n_static_faces) & (f != oracle.NO_FACE)).any())
    assert seen_vehicle


def test_channel_multi_equals_single(engine):
    """emrt_channel_multi (all frequencies in one pass) gives, frequency by
    frequency, exactly the outputs of emrt_channel."""
    sc = S.district_scene(seed=0)
    g = _gpu(engine, sc)
    p = g.trace(stride=61)
    assert p.n() > 50
    freqs = [3.5e9, 28e9, 5.9e9]
    multi = g.channels(p, freqs)
    for f, m in zip(freqs, multi):
        one = g.channel(p, f)
        n = p.n()
        assert torch.equal(m.path[:n], one.path[:n])
        assert torch.equal(m.pair, one.pair)
        assert torch.equal(m.rx, one.rx)


def test_constant_gamma_mode(engine):
    sc = S.toy_scene(seed=3)
    g = _gpu(engine, sc)
    p = g.trace(n_rays=50_000)
    ga = rec_to_paths(p.records())
    a, tau, fd, _ = _field(g, p, 3.5e9, const_gamma=True)
    o = oracle.OracleScene(sc, sc.frame(0), const_gamma=True)
    rf = compare_field(a, tau, fd, *oracle.field(o, ga, 3.5e9))
    assert rf["ok"], rf


def test_edge_cases(engine):
    E = engine
    # K = 0 (line of sight only), single receiver, ragged ray count
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    fr1 = dataclasses.replace(fr, rx_pos=fr.rx_pos[:1], rx_vel=fr.rx_vel[:1])
    g = _gpu(E, sc, fr1)
    p = g.trace(n_rays=12_345, max_depth=0, count=1001)
    ga = rec_to_paths(p.records())
    assert (ga["depth"] == 0).all() and len(ga) <= 1
    o = oracle.OracleScene(sc, fr1)
    assert len(ga) == len(oracle.enumerate_paths(o, 0))
    # no static faces at all
    sc2 = S.custom_scene([], [], (0, 0, 5), [(10, 0, 5), (0, 30, 1)])
    g2 = _gpu(E, sc2)
    p2 = g2.trace(n_rays=10_000, max_depth=4)
    assert p2.n() == 2
    # capacity error surfaces through emrt_sync with the required count
    g3 = _gpu(E, sc)
    small = E.Paths(2, g3.device)
    g3.trace_async(small, n_rays=100_000, max_depth=2)
    with pytest.raises(E.N.EmrtError) as ei:
        g3.sync()
    assert ei.value.code == 4
    assert small.n() > 2


@pytest.mark.parametrize("form", ["depth_first", "breadth_first", "static_cache"])
def test_dense_receiver_cluster(engine, form):
    """Segments whose reception spheres hold more receivers than the merged
    query buffers (64) take the receiver-tree query instead; the detections
    are the oracle's either way.  A cube of 1000 receivers 20 m from the
    transmitter, 5000 rays (sphere radius ~0.8 m there): the rays through it
    detect ~200 receivers each."""
    E = engine
    rng = np.random.default_rng(3)
    rx = np.column_stack([rng.uniform(18.5, 21.5, 1000), rng.uniform(-1.5, 1.5, 1000),
                          rng.uniform(0.5, 3.5, 1000)])
    sc = S.custom_scene([S.rect_xy(-60, -60, 60, 60)], [0], (0, 0, 10), rx, n_rays=5000,
                        depth=1)
    g = _gpu(E, sc)
    p = g.trace(keep_rejected=True, breadth_first=form == "breadth_first",
                static_cache=form == "static_cache")
    st = g.last_stats
    assert st["rx_node_visits"] > 0, st  # the receiver-tree query ran
    o = oracle.OracleScene(sc, sc.frame(0))
    gu = rec_to_paths(p.records())
    cands, ray_marg, _ = oracle.trace(o, sc.n_rays, sc.max_depth)
    assert len(cands) > 500
    rc = compare_candidates(gu, cands, ray_marg)
    assert not rc["missing"] and not rc["extra_bad"], rc
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra


@pytest.mark.parametrize("n_small,clustered", [(4096, False), (65536, False), (4096, True),
                                               (65536, True)])
def test_tree_builders_agree_at_the_size_threshold(engine, n_small, clustered):
    """Per-frame trees of up to 4096 primitives are built by one block, up to
    65536 by one cooperative launch, larger ones by the device-wide path; the
    trees may differ but every query is exact, so the paths of n_small
    receivers are the same whether one more receiver (which moves the
    receiver and merged trees to the next builder) is present or not.
    Clustered: half of the receivers in one 0.5 m cube, so that many share a
    Morton code and the sorts' ties (by index) decide the trees."""
    E = engine
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    rng = np.random.default_rng(9)
    m = n_small + 1
    rx = np.column_stack([rng.uniform(-90, 90, m), rng.uniform(-90, 90, m),
                          rng.uniform(1.0, 3.0, m)]).astype(np.float32)
    if clustered:
        h = m // 2
        rx[:h] = (np.array([12.0, -7.0, 1.5]) + rng.uniform(0, 0.5, (h, 3))).astype(np.float32)
    big = dataclasses.replace(fr, rx_pos=rx, rx_vel=np.zeros_like(rx))
    small = dataclasses.replace(fr, rx_pos=rx[:n_small], rx_vel=np.zeros_like(rx[:n_small]))
    g = _gpu(E, sc, big, max_rx=m)
    rb = g.trace(n_rays=50_000).records()
    g.update(small)
    rs = g.trace(n_rays=50_000).records()
    keep = rb[rb[:, 1] < n_small]
    assert len(rs) > 1000
    assert np.array_equal(keep, rs)


def test_invalid_arguments(engine):
    E = engine
    sc = S.toy_scene(seed=0)
    g = E.Scene(sc)
    out = E.Paths(16, g.device)
    with pytest.raises(E.N.EmrtError) as ei:   # trace before any update
        g.trace_async(out)
    assert ei.value.code == 6
    g.update(sc.frame(0))
    with pytest.raises(E.N.EmrtError) as ei:
        g.trace_async(out, max_depth=5)
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:
        g.trace_async(out, stride=0)
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:
        g.trace_async(out, n_rays=100, offset=100)
    assert ei.value.code == 1
    # multi-frequency channel: 1..8 frequencies, all positive
    paths = g.trace(n_rays=20_000)
    with pytest.raises(E.N.EmrtError) as ei:
        g.channels(paths, [])
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:
        g.channels(paths, [3.5e9] * 9)
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:
        g.channels(paths, [3.5e9, -1.0])
    assert ei.value.code == 1
    # a non-finite material parameter surfaces as a device error at the next
    # sync (host-injected fault); the error word is cleared by that sync
    nan_eps = g.eps_r.clone()
    nan_eps.fill_(float("nan"))
    g.channel(paths, 3.5e9, eps_r=nan_eps)
    with pytest.raises(E.N.EmrtError) as ei:
        g.sync()
    assert ei.value.code == 7
    g.channel(paths, 3.5e9)
    g.sync()
    # the same for the adjoint: NaN materials give NaN tangents, reported at
    # the next sync
    cot = torch.ones((g.n_tx, g.n_rx, 2), dtype=torch.float64, device=g.device)
    g.channel_backward(paths, 3.5e9, cot, eps_r=nan_eps)
    with pytest.raises(E.N.EmrtError) as ei:
        g.sync()
    assert ei.value.code == 7
    g.channel_backward(paths, 3.5e9, cot)
    g.sync()
    # rediscovery does not keep rejected candidates
    p = E.N.TraceParams(2, 20_000, 0, 1, 0, E.N.TRACE_KEEP_REJECTED)
    pc = paths.c()
    code = g.lib.emrt_rediscover(g.h, E.C.byref(p), E.C.byref(pc), None)
    assert code == 1
