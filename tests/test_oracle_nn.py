"""Pins of the network reference (CPU): convolution against scipy's correlation,
the identity kernel, adjointness of pooling and upsampling, and every gradient
against central finite differences."""
import numpy as np
import pytest

from oracle import nn


def rand_params(rng, scale=0.2):
    return [(rng.standard_normal((3, 3, 3, ci, co)) * scale / np.sqrt(27 * ci),
             rng.standard_normal(co) * 0.05) for ci, co in nn.LAYERS]


def test_conv_matches_scipy_correlate():
    scipy_nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 6, 8, 3))
    w = rng.standard_normal((3, 3, 3, 3, 2))
    b = rng.standard_normal(2)
    out = nn.conv3d(x, w, b)
    for co in range(2):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            xp = np.pad(x[..., ci], ((1, 1), (0, 0), (0, 0)))      # zeros in z
            full = scipy_nd.correlate(xp, w[:, :, :, ci, co], mode="wrap")
            ref += full[1:-1]
        assert np.allclose(out[..., co], ref, rtol=1e-12, atol=1e-12)


def test_identity_kernel_copies():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 4, 5))
    w = np.zeros((3, 3, 3, 5, 5))
    w[1, 1, 1] = np.eye(5)
    assert np.array_equal(nn.conv3d(x, w, np.zeros(5)), x)


def test_pool_up_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 6, 8, 3))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(nn.pool2(x) * y), np.sum(x * nn.pool2_backward(y)))
    assert np.isclose(np.sum(nn.up2(y) * x), np.sum(y * nn.up2_backward(x)))


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    params = rand_params(rng, scale=1.0)
    x = rng.standard_normal((4, 4, 4, nn.CIN))
    t = rng.standard_normal((4, 4, 4))

    def loss(ps):
        return nn.mse(nn.forward(ps, x)[0], t)[0]

    y, cache = nn.forward(params, x)
    _, dy = nn.mse(y, t)
    grads = nn.backward(params, cache, dy)
    h = 1e-6
    for layer in range(6):
        for which in (0, 1):
            arr = params[layer][which]
            for _ in range(4):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                orig = arr[idx]
                arr[idx] = orig + h
                lp = loss(params)
                arr[idx] = orig - h
                lm = loss(params)
                arr[idx] = orig
                fd = (lp - lm) / (2 * h)
                an = grads[layer][which][idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (layer, which, fd, an)


def test_adam_first_step_moves_by_lr_times_sign():
    """Adam's bias-corrected first step is lr * g / (|g| + eps) (Kingma & Ba)."""
    rng = np.random.default_rng(4)
    params = rand_params(rng)
    grads = [(rng.standard_normal(w.shape), rng.standard_normal(b.shape)) for w, b in params]
    m = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
    v = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
    new = nn.adam(params, grads, m, v, 1, lr=1e-3)
    for (w, b), (w2, b2), (dw, db) in zip(params, new, grads):
        assert np.allclose(w - w2, 1e-3 * dw / (np.abs(dw) + 1e-8), rtol=1e-10)
