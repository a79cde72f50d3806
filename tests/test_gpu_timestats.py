"""Eq. 1 correlation and Eq. 2 coherence time: CUDA against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_correlation_and_coherence_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    # channel series of the district over 24 frames (coherent sums per pair)
    sc = S.district_scene(seed=6)
    g = engine.Scene(sc)
    series = []
    for k in range(24):
        g.update(sc.frame(k))
        p = g.trace(stride=13)
        series.append(g.channel(p, 3.5e9).pair[..., :2].reshape(-1, 2).clone())
    h = torch.stack(series)                       # [F, P, 2]
    R = engine.channel_correlation(h, 10).cpu().numpy()
    hn = h.cpu().numpy()
    R_o = oracle.channel_correlation(hn[..., 0] + 1j * hn[..., 1], 10)
    assert R == pytest.approx(R_o, abs=1e-9)
    assert np.all(R[:, 0][np.abs(R_o[:, 0]) > 0] == pytest.approx(1.0))
    # coherence time of the last frame
    fr = sc.frame(23)
    tc = g.coherence_time(3.5e9, 0.5).cpu().numpy()
    tc_o = oracle.coherence_time(fr.tx_pos, fr.rx_pos, fr.rx_vel, 3.5e9, 0.5)
    fin = np.isfinite(tc_o)
    assert np.array_equal(fin, np.isfinite(tc))
    assert tc[fin] == pytest.approx(tc_o[fin], rel=1e-9)
    assert g.refresh_interval(3.5e9, sc.dt) >= 1
