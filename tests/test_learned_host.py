"""Host-side logic of the learned guess's training set-up (no GPU): the
extrapolation start of the network is exactly linear extrapolation in time,
checked with the FP64 CNN oracle, and keeps free channels for training."""
import numpy as np
import pytest

import paper_2305_13555_gb300 as pkg
from oracle import nn as onn
from paper_2305_13555_gb300 import build as pbuild
from paper_2305_13555_gb300 import learned


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pbuild.build()
    pkg.load_library()


def test_extrapolation_start_is_linear_extrapolation():
    """out = input channels 4-7 (the last step's normalised change), so
    phi_hat = phi_{n-1} + S out = 2 phi_{n-1} - phi_{n-2}, at every cell
    including the slab ends, whatever the other inputs are."""
    g = np.random.default_rng(5)
    theta = learned.extrapolation_params(seed=3).astype(np.float64)
    x = g.normal(0, 1, (3, 13, 37))
    out, _ = onn.forward(theta, x)
    assert np.array_equal(out, x[:, 4:8])


def test_extrapolation_start_leaves_channels_free():
    """Channels 8-31 of layers 1-4 start random (something to train), the
    last layer reads channels 0-7 only, and the weights are exact in BF16
    (0 and +-1), so the GPU's BF16 rounding keeps the start exact."""
    theta = learned.extrapolation_params(seed=3)
    layers = onn.unflatten(theta.astype(np.float64))
    for l, (W, b) in enumerate(layers[:-1]):
        assert np.count_nonzero(W[8:]) > 0.9 * W[8:].size, l
        assert not np.any(b)
    W4, b4 = layers[-1]
    assert not np.any(W4[:, 8:]) and not np.any(b4)
    for W, _ in layers:
        assert set(np.unique(W[:8] if W.shape[0] > 4 else W)) <= {-1.0, 0.0, 1.0}
