"""The field stage as a torch.autograd.Function (EMFieldFn): a torch loss over
received power, differentiated through the hand-written adjoint, against
central finite differences of the FP64 oracle (district frozen at frame 0,
8 materials, 2 transmitters), and torch.autograd.gradcheck on the material
parameters."""
import numpy as np
import pytest

import oracle
from helpers import rec_to_paths
from paper_2303_10521_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_10521_gb300 import engine, autograd
    sc = S.district_scene(seed=4)
    fr = sc.frame(0)
    g = engine.Scene(sc)
    g.update(fr)
    paths = g.trace(stride=7)
    return sc, fr, g, paths, autograd


def test_loss_backward_matches_oracle_finite_differences(setup):
    sc, fr, g, paths, AG = setup
    ga = rec_to_paths(paths.records())
    assert len(ga) > 50
    f, pt = sc.freqs[0], sc.tx_power_w
    dev = g.device
    eps = torch.tensor(sc.eps_r, dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(sc.sigma, dtype=torch.float64, device=dev, requires_grad=True)
    txp = torch.tensor(fr.tx_pos, dtype=torch.float64, device=dev, requires_grad=True)
    h = AG.EMFieldFn.apply(eps, sig, txp, g, paths, f)
    p = pt * (h ** 2).sum(-1).sum(0)
    mask = p > 0
    rng = np.random.default_rng(5)
    p_np = p.detach().cpu().numpy()
    m_np = mask.cpu().numpy()
    target = 10 * np.log10(np.where(m_np, p_np, 1.0) * 1e3) + rng.normal(0, 3, len(p_np))
    tgt = torch.as_tensor(target, device=dev)
    dbm = 10 * torch.log10(torch.where(mask, p, torch.ones_like(p)) * 1e3)
    loss = (torch.where(mask, dbm - tgt, torch.zeros_like(p)) ** 2).sum()
    loss.backward()
    fe, fs, ft = oracle.fd_gradient(sc, fr, ga, f, pt, target, m_np)
    for got, want in ((eps.grad, fe), (sig.grad, fs), (txp.grad, ft)):
        got = got.cpu().numpy().ravel()
        want = np.asarray(want).ravel()
        scale = np.abs(want).max()
        assert scale > 0
        assert np.all(np.abs(got - want) <= 1e-3 * np.maximum(np.abs(want), 1e-3 * scale)), \
            (got, want)


def test_gradcheck_material_parameters(setup):
    sc, fr, g, paths, AG = setup
    f = sc.freqs[0]
    dev = g.device
    txp = torch.tensor(fr.tx_pos, dtype=torch.float64, device=dev)
    h0 = AG.EMFieldFn.apply(torch.tensor(sc.eps_r, dtype=torch.float64, device=dev),
                            torch.tensor(sc.sigma, dtype=torch.float64, device=dev), txp, g,
                            paths, f)
    w = torch.randn(h0.shape, dtype=torch.float64, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(3)) / h0.abs().max()
    eps = torch.tensor(sc.eps_r, dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(sc.sigma, dtype=torch.float64, device=dev, requires_grad=True)
    fn = lambda e, s: (AG.EMFieldFn.apply(e, s, txp, g, paths, f) * w).sum()
    assert torch.autograd.gradcheck(fn, (eps, sig), eps=1e-6, atol=1e-6, rtol=1e-3)
