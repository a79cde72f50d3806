"""Per-receiver re-discovery schedule through the C-ABI against the oracle's
rule, frame by frame (integer decisions: bit-exact), and the cached frame it
drives (revalidation + backward re-discovery of the due receivers)."""
import numpy as np
import pytest

import oracle
from helpers import rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine as E
    return E


@pytest.mark.parametrize("dt,d_seg,max_interval", [(0.1, 10.0, 50), (0.0, 3.0, 6)])
def test_schedule_matches_oracle(engine, dt, d_seg, max_interval):
    sc = S.district_scene(seed=2)
    g = engine.Scene(sc)
    fr = sc.frame(0)
    g.update(fr)
    sched = engine.RefreshSchedule(g.n_tx, g.n_rx, g.device, freq=3.5e9, dt=dt, d_seg=d_seg,
                                   max_interval=max_interval)
    st = np.full((g.n_rx, 4), -1.0, np.float32)
    ref = np.zeros((g.n_tx, g.n_rx), np.uint8)
    n_seen = []
    for k in range(0, 40, 3):
        fr = sc.frame(k)
        g.update(fr)
        g.refresh_schedule(sched)
        due = sched.due().cpu().numpy()
        o = oracle.OracleScene(sc, fr)
        due_o, st, ref = oracle.refresh_schedule(o, st, ref, 3.5e9, 0.5, dt, d_seg,
                                                 max_interval)
        diff = sorted(set(due.tolist()) ^ set(due_o.tolist()))
        if diff:  # only where a line of sight lies within the acceptance margin
            direct = np.zeros(g.n_tx * g.n_rx, oracle.PATH_DTYPE)
            direct["tx"] = np.repeat(np.arange(g.n_tx), g.n_rx)
            direct["rx"] = np.tile(np.arange(g.n_rx), g.n_tx)
            direct["face"] = oracle.NO_FACE
            _, marg = oracle.validate(o, direct)
            marg = marg.reshape(g.n_tx, g.n_rx)
            assert all((marg[:, r] != 0).any() for r in diff), (k, diff)
            st, ref = sched.state.cpu().numpy(), sched.los_ref.cpu().numpy()
        assert np.array_equal(sched.state.cpu().numpy(), st), k
        assert np.array_equal(sched.los_ref.cpu().numpy(), ref), k
        n_seen.append(len(due))
    assert n_seen[0] == g.n_rx and 0 < min(n_seen[1:]) and max(n_seen[1:]) < g.n_rx


def test_cached_frame_with_backward_refresh(engine):
    """Revalidated cache + backward re-discovery of the due receivers: every
    kept path is valid for the oracle, and the due receivers' paths contain
    what a full backward trace of those receivers accepts."""
    sc = S.district_scene(seed=3)
    g = engine.Scene(sc)
    g.update(sc.frame(0))
    cache = g.trace(stride=17)
    sched = engine.RefreshSchedule(g.n_tx, g.n_rx, g.device, freq=3.5e9, dt=0.0, d_seg=4.0,
                                   max_interval=20)
    g.refresh_schedule(sched)                      # frame 0: everyone
    fr = sc.frame(6)
    g.update(fr)
    g.revalidate(cache)
    g.refresh_schedule(sched)
    ids = sched.due()
    assert 0 < len(ids) < g.n_rx
    fresh = g.trace_backward(ids, n_rays=200_000)
    g.merge(cache, fresh)
    got = rec_to_paths(cache.records())
    o = oracle.OracleScene(sc, fr)
    acc, marg = oracle.validate(o, got)
    assert (acc | (marg != 0)).all()
    kf = {tuple(r) for r in oracle.key_fields(rec_to_paths(fresh.records())).tolist()}
    kc = {tuple(r) for r in oracle.key_fields(got).tolist()}
    assert kf <= kc and set(rec_to_paths(fresh.records())["rx"].tolist()) <= set(
        ids.cpu().tolist())
