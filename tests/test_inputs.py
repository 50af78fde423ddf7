"""Host-side checks of the seeded synthetic inputs (no solver arithmetic)."""
import math

import numpy as np

from paper_1410_8568_gb300 import inputs as I


def test_config1_geometry_and_rhs():
    P = I.config1(32)
    assert P.shape == (32, 32, 32) and P.bc == (0, 0, 0)
    assert P.rho.shape == (32, 32, 32)
    assert abs(P.rho[16, 16, 16] - 1000.0) < 1.0  # centre of the sphere is liquid (tanh tail)
    assert abs(P.rho[0, 0, 0] - 1.0) < 1e-3
    assert abs(P.rhs.mean()) < 1e-15
    Q = I.config1(32)
    assert np.array_equal(P.rhs, Q.rhs) and np.array_equal(P.rho, Q.rho)


def test_drop_film_geometry():
    P = I.config2(64)
    assert P.bc == (1, 1, 0)
    assert abs(P.rho[0, 10, 10] - 1000.0) < 1.0  # bottom film
    k = int(0.3 * 64)
    assert abs(P.rho[k, 32, 32] - 1000.0) < 1.0  # drop centre
    assert abs(P.rho[-1, 0, 0] - 1.0) < 1e-3  # gas above
    assert P.rho.min() >= 1.0 - 1e-12 and P.rho.max() <= 1000.0 + 1e-9


def test_fourier_divergence_telescopes():
    rng = np.random.default_rng(0)
    for bc in [(1, 1, 0), (0, 0, 0), (1, 1, 1)]:
        b = I.rhs_fourier_divergence((16, 12, 8), bc, np.random.default_rng(3), zchunk=3)
        b2 = I.rhs_fourier_divergence((16, 12, 8), bc, np.random.default_rng(3), zchunk=64)
        assert np.allclose(b, b2, rtol=0, atol=1e-12)
        assert abs(b.mean()) < 1e-13
        assert np.abs(b).max() > 1.0
    del rng


def test_batch_and_stream_are_seeded():
    a = I.config4_batch(6)
    b = I.config4_batch(6)
    for p, q in zip(a, b):
        assert p.shape == q.shape and np.array_equal(p.rhs, q.rhs)
        assert p.shape[0] in I.BATCH_EDGES and p.ratio in (10.0, 100.0, 1000.0)
    s = I.config5_stream(50, rate=3.0)
    assert s == I.config5_stream(50, rate=3.0)
    assert all(e in I.STREAM_EDGES for _, e, _, _ in s)
    t = [r[0] for r in s]
    assert all(t2 > t1 for t1, t2 in zip(t, t[1:]))
    assert all(10.0 <= r[2] <= 1000.0 for r in s)


def test_config3_droplets_in_gas():
    rng = np.random.default_rng(5)
    d = I._gas_droplets(rng, 4)
    for (c, r) in d:
        assert 0.02 <= r <= 0.05
        assert c[2] - r > 0.1
        assert math.dist(c, (0.5, 0.5, 0.3)) > 0.125 + r
