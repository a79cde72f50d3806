"""Parity at the benchmark's full size and launch configuration: the 2x2 km
city (293k triangles, 5000 vehicles, 10k receivers, 4 transmitters x 1e7
rays, 4 reflections, reflected rays sorted between bounces).

* acceptance: every unique candidate of the full trace is re-validated by
  the oracle (image method + brute-force occlusion); flags must agree except
  where the oracle reports a margin;
* field and reduction: every accepted path, element by element, and every
  (tx, rx) pair;
* discovery: the oracle traces an evenly spaced sample of the rays; every
  candidate it finds outside the margin must be among the GPU's unique
  candidates, and every GPU candidate whose recorded ray is in the sample
  must be an oracle candidate of that ray set or come from a marginal ray.
"""
import numpy as np
import pytest

import oracle
from helpers import compare_acceptance, compare_field, rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_ABS, EPS_REL = 1e-4, 2e-7   # margin: 1e-4 m plus float32 drift over the path


@pytest.fixture(scope="module")
def city():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    sc = S.city_scene(seed=0)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    allc = g.trace(keep_rejected=True)
    acc = g.trace()
    return sc, fr, g, allc, acc, oracle.OracleScene(sc, fr)


def test_city_depth_first_equals_breadth_first(city):
    """Full-size city frame: the default depth-first chains and the
    breadth-first form with the coherence sort give the same records."""
    sc, fr, g, allc, acc, o = city
    b = g.trace(keep_rejected=True, breadth_first=True, sort_rays=True).records()
    assert np.array_equal(b, allc.records())


def test_city_wide_bvh_identical(city):
    """Full-size city frame through the compressed 8-wide tree (8-bit child
    boxes), depth-first and breadth-first: the binary tree's records and
    segments, bit for bit; fewer node fetches per segment."""
    sc, fr, g, allc, acc, o = city
    g.trace(keep_rejected=True)
    s2 = dict(g.last_stats)
    for kw in (dict(), dict(breadth_first=True)):
        w = g.trace(keep_rejected=True, wide_bvh=True, **kw).records()
        s8 = dict(g.last_stats)
        assert np.array_equal(w, allc.records()), kw
        assert s8["segments"] == s2["segments"], kw
        assert s8["node_visits"] < 0.7 * s2["node_visits"], (s8["node_visits"], s2["node_visits"])


def test_city_acceptance_every_candidate(city):
    sc, fr, g, allc, acc, o = city
    gu = rec_to_paths(allc.records())
    assert len(gu) > 10_000
    r = compare_acceptance(o, gu, eps_abs=EPS_ABS, eps_rel=EPS_REL)
    assert r["n_diff_unflagged"] == 0, {k: v for k, v in r.items() if k != "bad"}
    assert len(rec_to_paths(acc.records())) == r["n_acc_gpu"]


def test_city_field_and_reduction_every_path(city):
    sc, fr, g, allc, acc, o = city
    ga = rec_to_paths(acc.records())
    for f in sc.freqs:
        ch = g.channel(acc, f)
        n = acc.n()
        po = ch.path[:n].cpu().numpy()
        a_o, tau_o, fd_o = oracle.field(o, ga, f)
        r = compare_field(po[:, 0] + 1j * po[:, 1], po[:, 2], po[:, 3], a_o, tau_o, fd_o)
        assert r["ok"], (f, r)
        st = oracle.reduce(ga, a_o, tau_o, fd_o, len(fr.tx_pos), len(fr.rx_pos))
        pair = ch.pair.cpu().numpy()
        sum_abs = np.zeros(st.shape[:2])
        np.add.at(sum_abs, (ga["tx"].astype(int), ga["rx"].astype(int)), np.abs(a_o))
        h_err = np.abs(pair[..., 0] + 1j * pair[..., 1] - (st[..., 0] + 1j * st[..., 1]))
        assert np.all(h_err <= 1e-4 * sum_abs + 1e-30)
        assert np.array_equal(pair[..., 7], st[..., 7])


def test_city_discovery_sampled_rays(city):
    sc, fr, g, allc, acc, o = city
    gu = rec_to_paths(allc.records())
    rng = np.random.default_rng(7)
    pick = rng.choice(len(gu), size=min(300, len(gu)), replace=False)
    rays = np.unique(np.concatenate([gu["ray"][pick].astype(np.uint64),
                                     np.arange(0, sc.n_rays, 50_000, dtype=np.uint64)]))
    cands, ray_marg, _ = oracle.trace_list(o, sc.n_rays, sc.max_depth, rays,
                                           eps_abs=EPS_ABS, eps_rel=EPS_REL)
    cands["ray"] = rays[cands["ray"]].astype(np.uint32)     # back to ray indices
    ou = oracle.dedup(cands)
    gkeys = {tuple(k) for k in oracle.key_fields(gu)}
    okeys = {tuple(k): int(f) for k, f in zip(oracle.key_fields(ou), ou["flag"])}
    missing = [k for k, f in okeys.items() if f == 0 and k not in gkeys]
    assert not missing, missing[:5]
    where = {int(r): i for i, r in enumerate(rays)}
    bad, checked = [], 0
    for k, p in zip(oracle.key_fields(gu), gu):
        j = int(p["ray"])
        if j not in where:
            continue
        checked += 1
        if tuple(k) in okeys:
            continue
        if ray_marg[int(p["tx"]), where[j]] > int(p["depth"]):
            bad.append(tuple(k))
    assert not bad, bad[:5]
    assert checked >= 250 and len(okeys) >= 250


def test_city_static_cache_identical(city):
    """The static-hit cache gives the plain trace's unique candidates bit for
    bit at the benchmark size, on the cold frame and two frames later."""
    sc, fr, g, allc, acc, o = city
    ref = allc.records()
    cold = g.trace(keep_rejected=True, sort_rays=True, static_cache=True).records()
    assert np.array_equal(ref, cold)
    for k in (2,):
        g.update(sc.frame(k))
        a = g.trace(keep_rejected=True, sort_rays=True).records()
        sa = dict(g.last_stats)
        b = g.trace(keep_rejected=True, sort_rays=True, static_cache=True).records()
        sb = dict(g.last_stats)
        assert np.array_equal(a, b)
        assert sa["segments"] == sb["segments"]
        assert sb["static_reused"] > 0.9 * sum(sb["segments"])
    g.update(fr)
