"""Backward (receiver-side) discovery, Sec. II-A, through the C-ABI: parity
with the oracle's role-exchanged discovery, record by record, and
reciprocity with forward discovery."""
import dataclasses

import numpy as np
import pytest

import oracle
from helpers import compare_acceptance, compare_candidates, compare_field, rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine as E
    return E


def _ids(g, ids):
    return None if ids is None else torch.tensor(ids, dtype=torch.int32, device=g.device)


def test_toy_backward_parity(engine):
    """Toy scene, every receiver shoots N = 1e5 rays, K = 2."""
    sc = S.toy_scene(seed=0)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    o = oracle.OracleScene(sc, fr)
    allc = g.trace_backward(keep_rejected=True)
    gu = rec_to_paths(allc.records())
    cands, marg, _ = oracle.trace_backward(sc, fr, sc.n_rays, sc.max_depth)
    rows = {r: r for r in range(len(fr.rx_pos))}
    rc = compare_candidates(gu, cands, marg, rx_rows=rows)
    assert not rc["missing"] and not rc["extra_bad"], rc
    assert rc["n_gpu"] > 20
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra
    acc = g.trace_backward()
    ga = rec_to_paths(acc.records())
    assert len(ga) == ra["n_acc_gpu"]
    k = oracle.key_fields(ga)
    assert all(tuple(k[i]) < tuple(k[i + 1]) for i in range(len(k) - 1))
    ch = g.channel(acc, sc.freqs[0])
    po = ch.path[:acc.n()].cpu().numpy()
    rf = compare_field(po[:, 0] + 1j * po[:, 1], po[:, 2], po[:, 3],
                       *oracle.field(o, ga, sc.freqs[0]))
    assert rf["ok"], rf


def test_backward_subset_and_reciprocity(engine):
    """A receiver subset gives exactly the full backward records of those
    receivers; backward and forward discovery agree with the exhaustive
    enumeration (reciprocal paths)."""
    sc = S.toy_scene(seed=1)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    ids = [1, 4, 9, 14]
    full = g.trace_backward().records()
    sub = g.trace_backward(_ids(g, ids)).records()
    ref = full[np.isin(full[:, 1], ids)]
    assert len(ref) > 5 and np.array_equal(sub, ref)
    o = oracle.OracleScene(sc, fr)
    exact = oracle.enumerate_paths(o, sc.max_depth)
    a, _, _ = oracle.field(o, exact, sc.freqs[0])
    w = dict(zip(map(tuple, oracle.key_fields(exact).tolist()), np.abs(a) ** 2))
    tot = sum(w.values())
    fwd = {tuple(r) for r in oracle.key_fields(rec_to_paths(g.trace().records())).tolist()}
    bwd = {tuple(r) for r in oracle.key_fields(rec_to_paths(full)).tolist()}
    assert bwd <= set(w) and fwd <= set(w)
    assert sum(w[k] for k in bwd) / tot > 0.99
    assert sum(w[k] for k in fwd & bwd) / tot > 0.98


def test_district_backward_subsample_parity(engine):
    """District (400 buildings, 200 vehicles, K = 3): 8 receivers shoot a
    strided subset of the 1M rays on both sides."""
    sc = S.district_scene(seed=0)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    o = oracle.OracleScene(sc, fr)
    ids = [3, 100, 257, 400, 512, 640, 777, 999]
    stride, offset = 409, 7
    allc = g.trace_backward(_ids(g, ids), stride=stride, offset=offset, keep_rejected=True)
    gu = rec_to_paths(allc.records())
    assert set(gu["rx"].tolist()) <= set(ids)
    cands, marg, _ = oracle.trace_backward(sc, fr, sc.n_rays, sc.max_depth, rx_ids=ids,
                                           offset=offset, stride=stride)
    rc = compare_candidates(gu, cands, marg, rx_rows={r: i for i, r in enumerate(ids)})
    assert not rc["missing"] and not rc["extra_bad"], {k: v for k, v in rc.items() if k != "bad"}
    ra = compare_acceptance(o, gu)
    assert ra["n_diff_unflagged"] == 0, ra


def test_backward_invalid_arguments(engine):
    E = engine
    sc = S.toy_scene(seed=0)
    g = E.Scene(sc)
    g.update(sc.frame(0))
    out = E.Paths(64, g.device)
    with pytest.raises(E.N.EmrtError) as ei:   # empty receiver list
        g.trace_backward_async(out, torch.zeros(0, dtype=torch.int32, device=g.device))
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:   # more sources than receivers
        g.trace_backward_async(out, torch.zeros(17, dtype=torch.int32, device=g.device))
    assert ei.value.code == 1
    with pytest.raises(E.N.EmrtError) as ei:   # ray count above the id bits (16 Rx: 28)
        g.trace_backward_async(out, n_rays=(1 << 28) + 2, max_depth=1)
    assert ei.value.code == 1
    # K = 0: line of sight only, from one receiver
    fr1 = dataclasses.replace(sc.frame(0))
    g.update(fr1)
    p = g.trace_backward(_ids(g, [7]), n_rays=20_000, max_depth=0)
    ga = rec_to_paths(p.records())
    o = oracle.OracleScene(sc, fr1)
    ex = oracle.enumerate_paths(o, 0)
    assert ga["rx"].tolist() == ex["rx"][ex["rx"] == 7].tolist()
