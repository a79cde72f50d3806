"""Adjoint of the field stage (emrt_channel_backward) against central finite
differences of the FP64 oracle, on the district scene frozen at frame 0
(8 materials, 2 transmitters, loss over received power in dBm)."""
import numpy as np
import pytest

import oracle
from helpers import rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dloss_dh(h, pt, target, mask):
    """Cotangent of loss = sum_mask (P_dBm - target)^2 w.r.t. (Re h, Im h)."""
    p = pt * (np.abs(h) ** 2).sum(0)
    dbm = 10 * np.log10(np.where(mask, p, 1.0) * 1e3)
    dl_dp = np.where(mask, 2 * (dbm - target) * 10 / (np.log(10) * np.where(mask, p, 1.0)), 0.0)
    g = np.zeros(h.shape + (2,))
    g[..., 0] = dl_dp[None, :] * 2 * pt * h.real
    g[..., 1] = dl_dp[None, :] * 2 * pt * h.imag
    return g


@pytest.mark.parametrize("stride", [7, 1])
def test_adjoint_matches_finite_differences(stride):
    """stride 1: the frozen full-density path topology of the differentiable
    field workload (1M rays per Tx, every path of frame 0); stride 7: a
    sparser topology of the same scene."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine
    sc = S.district_scene(seed=4)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    paths = g.trace(stride=stride)
    ga = rec_to_paths(paths.records())
    assert len(ga) > 50
    f = sc.freqs[0]
    ch = g.channel(paths, f)
    pair = ch.pair.cpu().numpy()
    h = pair[..., 0] + 1j * pair[..., 1]
    pt = sc.tx_power_w
    p0 = pt * (np.abs(h) ** 2).sum(0)
    mask = p0 > 0
    rng = np.random.default_rng(5)
    target = 10 * np.log10(np.where(mask, p0, 1.0) * 1e3) + rng.normal(0, 3, len(p0))
    cot = torch.as_tensor(_dloss_dh(h, pt, target, mask))
    ge, gs, gt = (t.cpu().numpy() for t in g.channel_backward(paths, f, cot))
    fe, fs, ft = oracle.fd_gradient(sc, fr, ga, f, pt, target, mask)
    if stride == 1:
        # full density: receivers near deep fades make the loss sharply
        # curved in the transmitter position, so the central difference's
        # O(h^2) error is removed by Richardson extrapolation over steps h
        # and 2h (error O(h^4)); the material steps need none
        _, _, ft2 = oracle.fd_gradient(sc, fr, ga, f, pt, target, mask, tx_h=2e-4)
        ft = (4.0 * ft - ft2) / 3.0
    for got, want in ((ge, fe), (gs, fs), (gt.ravel(), ft.ravel())):
        scale = np.abs(want).max()
        assert scale > 0
        err = np.abs(got - want)
        assert np.all(err <= 1e-3 * np.maximum(np.abs(want), 1e-3 * scale)), (got, want)
    # materials on no path have exactly zero gradient on both sides
    used = set()
    for p in ga:
        for q in range(int(p["depth"])):
            fc = int(p["face"][q])
            used.add(int(sc.face_mat[fc]) if fc < sc.n_static_faces else sc.veh_mat)
    for m in range(len(sc.eps_r)):
        if m not in used:
            assert ge[m] == 0 and gs[m] == 0
