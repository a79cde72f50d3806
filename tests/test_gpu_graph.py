"""Per-frame calls recorded into a caller's CUDA graph: a cached frame of the
district (update from one device pose buffer, rediscovery with revalidation
and the static-hit cache, fields at two frequencies) captured once and
replayed gives, frame after frame, the records and received powers of the
same calls issued one by one."""
import numpy as np
import pytest

from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("veh_pos", "veh_vel", "rx_pos", "rx_vel", "tx_pos", "tx_vel")


def test_cached_frame_graph_equals_eager():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    sc = S.district_scene(seed=2)
    dev = torch.device("cuda", 0)
    frames = [sc.frame(k) for k in range(6)]
    flat = torch.stack([torch.cat([torch.as_tensor(np.asarray(getattr(f, n), np.float32)).reshape(-1)
                                   for n in NAMES]) for f in frames]).to(dev)
    cur = torch.empty_like(flat[0])

    class F:
        pass

    v, o = F(), 0
    for n in NAMES:
        shp = np.asarray(getattr(frames[0], n)).shape
        m = int(np.prod(shp))
        setattr(v, n, cur[o:o + m].view(*shp))
        o += m
    g = engine.Scene(sc)
    cur.copy_(flat[0])
    g.update(v)
    cap = g.trace().capacity
    cache = engine.Paths(4 * cap, dev)
    chs = [None, None]
    freqs = [3.5e9, 28e9]

    def step():
        g.update(v)
        g.rediscover(cache, n_rays=sc.n_rays // 10, static_cache=True, revalidate=True)
        chs[:] = g.channels(cache, freqs, outs=chs)

    def restart():
        cur.copy_(flat[0])
        g.update(v)
        g.trace_async(cache, static_cache=True)
        g.sync()

    restart()
    for k in (1, 2):  # sizes every scratch buffer outside the capture
        cur.copy_(flat[k])
        step()
        g.sync()
    restart()
    eager = []
    for k in range(1, 6):
        cur.copy_(flat[k])
        step()
        g.sync()
        eager.append((cache.records(), chs[0].rx.clone(), chs[1].rx.clone()))
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, capture_error_mode="thread_local"):
        step()
    restart()
    for k in range(1, 6):
        cur.copy_(flat[k])
        gr.replay()
        st = g.sync()
        assert st["error_bits"] == 0
        rec, rx0, rx1 = eager[k - 1]
        assert len(rec) > 100
        assert np.array_equal(cache.records(), rec), k
        assert torch.equal(chs[0].rx, rx0) and torch.equal(chs[1].rx, rx1), k
