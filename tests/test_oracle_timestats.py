"""Pins of the oracle's channel statistics over time (Eq. 1 reading, Eq. 2)."""
import math

import numpy as np
import pytest

import oracle


def test_correlation_of_a_sinusoid_and_special_cases():
    F, period = 6000, 50
    t = np.arange(F)
    h = (2.0 + np.cos(2 * np.pi * t / period)) * np.exp(1j * 0.3 * t)   # |h| = 2 + cos
    R = oracle.channel_correlation(h[:, None], 60)[0]
    assert R[0] == pytest.approx(1.0, abs=1e-12)                        # any series
    assert R == pytest.approx(np.cos(2 * np.pi * np.arange(61) / period), abs=0.02)
    # constant magnitude: no fluctuation to correlate
    assert np.all(oracle.channel_correlation(np.exp(1j * t)[:, None], 5) == 0)
    # independent fluctuations decorrelate immediately
    rng = np.random.default_rng(3)
    Rn = oracle.channel_correlation((1 + rng.random(F))[:, None], 5)[0]
    assert abs(Rn[0] - 1) < 1e-12 and np.all(np.abs(Rn[1:]) < 0.05)


def test_coherence_time_eq2_properties():
    f = 3.5e9
    tx = [(0.0, 0.0, 30.0)]
    rx = [(100.0, 0.0, 1.5)]
    th = math.radians(60)
    v = [(10 * math.cos(math.pi - th), 10 * math.sin(math.pi - th), 0.0)]   # 60 deg off
    r = 2 ** -0.25                                      # sqrt(1/R^4 - 1) = 1
    k = np.array(rx[0]) - np.array(tx[0])
    theta = math.acos(np.dot(k, v[0]) / (np.linalg.norm(k) * 10.0))
    fd = f * 10.0 / oracle.C_LIGHT
    tc = oracle.coherence_time(tx, rx, v, f, r)[0, 0]
    assert tc == pytest.approx(1 / (2 * math.pi * fd * theta ** 2), rel=1e-12)
    # R = 1: no decorrelation allowed, zero coherence time
    assert oracle.coherence_time(tx, rx, v, f, 1.0)[0, 0] == 0.0
    # twice the speed, half the time; receiver at rest: unbounded
    v2 = [tuple(2 * np.array(v[0]))]
    assert oracle.coherence_time(tx, rx, v2, f, r)[0, 0] == pytest.approx(tc / 2, rel=1e-12)
    assert math.isinf(oracle.coherence_time(tx, rx, [(0, 0, 0)], f, r)[0, 0])
    # moving along the propagation direction: theta = 0, unbounded
    kk = tuple(k / np.linalg.norm(k) * 5)
    assert math.isinf(oracle.coherence_time(tx, rx, [kk], f, r)[0, 0])
