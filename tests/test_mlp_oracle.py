"""Pins of the FP64 reference of the learned-correction network."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_bf16_rounding_is_round_to_nearest_even():
    got = M.bf16(np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.14159265, -2.5e-3]))
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-8 -> 1 + 2^-6
    np.testing.assert_array_equal(got[:3], [1.0, 1.0, 1.0 + 2 ** -6])
    assert got[3] == 3.140625
    assert abs(got[4] / -2.5e-3 - 1) < 2 ** -8


def test_gelu_is_z_times_normal_cdf():
    for z in (-3.0, -0.5, 0.0, 0.7, 2.5):
        phi = 0.5 * math.erfc(-z / math.sqrt(2))
        assert abs(M.gelu(np.array(z)) - z * phi) < 1e-15
        h = 1e-6
        fd = (z + h) * 0.5 * math.erfc(-(z + h) / math.sqrt(2)) - (z - h) * 0.5 * math.erfc(-(z - h) / math.sqrt(2))
        assert abs(M.gelu_grad(np.array(z)) - fd / (2 * h)) < 1e-8


@pytest.mark.parametrize("n_in,H,n_out,batch", [(6, 5, 3, 7), (60, 16, 12, 9)])
def test_backward_matches_central_differences(n_in, H, n_out, batch):
    rng = np.random.default_rng(n_in)
    npar = H * n_in + H + H * H + H + n_out * H + n_out
    p = rng.normal(size=npar) * 0.4
    x = rng.normal(size=(batch, n_in))
    t = rng.normal(size=(batch, n_out))
    norm = (rng.normal(size=n_in), 1 + rng.random(n_in), rng.normal(size=n_out), 1 + rng.random(n_out))
    ident = lambda w: w  # noqa: E731  (finite differences need unrounded weights)
    _, g = M.loss_and_grad(p, x, t, norm, n_in, H, n_out, ident)
    eps = 1e-6
    idx = rng.choice(npar, size=min(npar, 60), replace=False)
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (M.loss_and_grad(pp, x, t, norm, n_in, H, n_out, ident)[0] -
              M.loss_and_grad(pm, x, t, norm, n_in, H, n_out, ident)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g).max()), (i, fd, g[i])
