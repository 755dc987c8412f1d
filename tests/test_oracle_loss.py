"""Pins of the oracle's squared-error loss (no GPU): closed forms and a central
finite-difference check of its gradient."""
import numpy as np

from oracle import oracle as O


def test_constant_offset_closed_form():
    rng = np.random.default_rng(0)
    t = rng.uniform(size=(37, 3))
    for delta in (0.0, 0.25, -1.5):
        loss, g = O.mse_loss(t + delta, t)
        assert abs(loss - delta * delta) <= 1e-15 * max(1.0, delta * delta)
        assert np.allclose(g, 2.0 * delta / t.size, rtol=0, atol=1e-15)


def test_hand_computed_small_case():
    loss, g = O.mse_loss(np.array([1.0, 2.0, 4.0]), np.array([0.0, 0.0, 0.0]))
    assert loss == (1.0 + 4.0 + 16.0) / 3.0
    assert np.array_equal(g, np.array([2.0, 4.0, 8.0]) / 3.0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    x, t = rng.normal(size=11), rng.normal(size=11)
    _, g = O.mse_loss(x, t)
    h = 1e-6
    for i in range(x.size):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (O.mse_loss(xp, t)[0] - O.mse_loss(xm, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-8


def test_empty():
    loss, g = O.mse_loss(np.zeros((0, 3)), np.zeros((0, 3)))
    assert loss == 0.0 and g.size == 0
