"""Pins of the FP64 MLP reference: GELU against z * Phi(z) from scipy's normal
CDF, and the hand-written gradient against central finite differences."""
import numpy as np
import pytest

from oracle import mlp as ref


def test_gelu_is_z_times_normal_cdf():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(ref.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(ref.gelu_grad(z), (ref.gelu(z + h) - ref.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n_in, hidden, B = 6, 5, 7
    n = hidden * n_in + hidden + 2 * (hidden * hidden + hidden) + hidden + 1
    p = rng.normal(0, 0.5, n)
    x = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, B)
    loss, g = ref.loss_and_grad(p, x, t, n_in, hidden)
    h = 1e-6
    for k in rng.choice(n, 25, replace=False):
        e = np.zeros(n)
        e[k] = h
        fd = (ref.loss_and_grad(p + e, x, t, n_in, hidden)[0] - ref.loss_and_grad(p - e, x, t, n_in, hidden)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
