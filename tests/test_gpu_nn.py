"""The network's BF16 tensor-core kernels against the FP64 oracle (oracle/nn.py).

The oracle takes the BF16-rounded weights and inputs, so the differences come
from BF16 storage of the intermediate activations and gradients (FP32
accumulation on the GPU); the bound is 2e-2 relative, normwise.
"""
import numpy as np
import pytest

from oracle import nn as onn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16_round(a):
    """Round-to-nearest-even of float32 values to bfloat16, returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def make(seed, D=4, H=8, W=8):
    from paper_2210_15668_gb300 import ferrox
    rng = np.random.default_rng(seed)
    ws, bs = ferrox.nn_init_params(seed)
    bs = [rng.standard_normal(b.shape) * 0.05 for b in bs]
    net = ferrox.NN(D, H, W, params=(ws, bs))
    x = bf16_round(rng.standard_normal((D, H, W, 16)))
    params = [(bf16_round(w).reshape(3, 3, 3, *w.shape[1:]), np.asarray(b, np.float32).astype(np.float64))
              for w, b in zip(ws, bs)]
    return net, x, params


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


@pytest.mark.parametrize("shape", [(4, 8, 8), (2, 6, 10), (8, 4, 16)])
def test_forward_matches_oracle(shape):
    net, x, params = make(1, *shape)
    y_or, _ = onn.forward(params, x)
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    y = net.forward(xt).cpu().numpy().reshape(shape)
    assert rel(y, y_or) <= 2e-2, rel(y, y_or)
    net.close()


def forward_backward_bf16_storage(params, x, t):
    """The oracle's layers composed with BF16 rounding wherever the GPU stores BF16
    (activations, upstream gradient, masked gradients); FP64 everywhere else."""
    r = bf16_round
    relu = lambda a: np.maximum(a, 0.0)  # noqa: E731
    a1 = r(relu(onn.conv3d(x, *params[0])))
    s1 = r(relu(onn.conv3d(a1, *params[1])))
    p = r(onn.pool2(s1))
    a3 = r(relu(onn.conv3d(p, *params[2])))
    a4 = r(relu(onn.conv3d(a3, *params[3])))
    cat = np.concatenate([onn.up2(a4), s1], axis=3)
    a5 = r(relu(onn.conv3d(cat, *params[4])))
    y = onn.conv3d(a5, *params[5])
    loss, dy0 = onn.mse(y[..., 0], t)
    dy = np.zeros_like(y)
    dy[..., 0] = dy0
    dy = r(dy)
    g = [None] * 6
    da5, *g[5] = onn.conv3d_backward(a5, params[5][0], dy)
    da5 = r(da5 * (a5 > 0))
    dcat, *g[4] = onn.conv3d_backward(cat, params[4][0], da5)
    da4 = r(onn.up2_backward(dcat[..., :32]) * (a4 > 0))
    da3, *g[3] = onn.conv3d_backward(a3, params[3][0], da4)
    da3 = r(da3 * (a3 > 0))
    dp, *g[2] = onn.conv3d_backward(p, params[2][0], da3)
    ds1 = r((dcat[..., 32:] + onn.pool2_backward(dp)) * (s1 > 0))
    da1, *g[1] = onn.conv3d_backward(a1, params[1][0], ds1)
    da1 = r(da1 * (a1 > 0))
    _, *g[0] = onn.conv3d_backward(x, params[0][0], da1)
    return loss, g


def test_gradients_match_oracle_with_bf16_storage():
    """Against the oracle's layers with BF16 storage emulated: 2e-2 normwise on every
    parameter gradient (the remaining differences are FP32 accumulation order)."""
    net, x, params = make(2, 4, 8, 8)
    t = np.random.default_rng(3).standard_normal((4, 8, 8))
    loss_or, g_or = forward_backward_bf16_storage(params, x, t)
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    tt = torch.as_tensor(t.ravel(), dtype=torch.float32, device="cuda")
    loss = net.loss_grad(xt, tt)
    _, _, gw, gb = net.params()
    assert abs(loss - loss_or) <= 2e-2 * loss_or
    for layer in range(6):
        e_w = rel(gw[layer], g_or[layer][0].reshape(27, *g_or[layer][0].shape[3:]))
        e_b = rel(gb[layer], g_or[layer][1])
        print(f"layer {layer}: grad rel err w {e_w:.2e} b {e_b:.2e}")
        assert e_w <= 2e-2 and e_b <= 2e-2, (layer, e_w, e_b)
    net.close()


def test_gradients_match_oracle():
    """Against the plain FP64 oracle (activations and gradients not rounded): the
    deepest layer's gradient passes through five BF16 roundings and ReLU masks of
    BF16 activations, so the bound here is 8e-2 normwise."""
    net, x, params = make(2, 4, 8, 8)
    rng = np.random.default_rng(3)
    t = rng.standard_normal((4, 8, 8))
    y_or, cache = onn.forward(params, x)
    loss_or, dy = onn.mse(y_or, t)
    g_or = onn.backward(params, cache, dy)
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    tt = torch.as_tensor(t.ravel(), dtype=torch.float32, device="cuda")
    loss = net.loss_grad(xt, tt)
    _, _, gw, gb = net.params()
    assert abs(loss - loss_or) <= 2e-2 * loss_or
    for layer in range(6):
        e_w = rel(gw[layer], g_or[layer][0].reshape(27, *g_or[layer][0].shape[3:]))
        e_b = rel(gb[layer], g_or[layer][1])
        print(f"layer {layer}: plain-oracle grad rel err w {e_w:.2e} b {e_b:.2e}")
        assert e_w <= 8e-2 and e_b <= 8e-2, (layer, e_w, e_b)
    net.close()


def test_adam_training_lowers_the_loss():
    net, x, params = make(4, 4, 8, 8)
    rng = np.random.default_rng(5)
    t = np.tanh(rng.standard_normal((4, 8, 8)))
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    tt = torch.as_tensor(t.ravel(), dtype=torch.float32, device="cuda")
    first = net.loss_grad(xt, tt)
    net.adam_step(1e-3)
    for _ in range(60):
        last = net.loss_grad(xt, tt)
        net.adam_step(1e-3)
    assert last < 0.5 * first, (first, last)
    net.close()


def forward_bf16_storage(params, x):
    """The oracle's forward with BF16 rounding wherever the GPU stores BF16 activations."""
    r = bf16_round
    relu = lambda a: np.maximum(a, 0.0)  # noqa: E731
    a1 = r(relu(onn.conv3d(x, *params[0])))
    s1 = r(relu(onn.conv3d(a1, *params[1])))
    p = r(onn.pool2(s1))
    a3 = r(relu(onn.conv3d(p, *params[2])))
    a4 = r(relu(onn.conv3d(a3, *params[3])))
    cat = np.concatenate([onn.up2(a4), s1], axis=3)
    a5 = r(relu(onn.conv3d(cat, *params[4])))
    return onn.conv3d(a5, *params[5])[..., 0]


# (grid, convolutions of the forward pass on the tcgen05 kernel): the fine grid
# needs x % 8 == 0 and y % 16 == 0, the pooled grid the same; (16, 128, 128) runs
# four z-planes per CTA on the fine grid, (6, 32, 16) an odd pooled depth
TC_SHAPES = [((4, 32, 16), 6), ((6, 32, 16), 6), ((4, 16, 8), 4), ((16, 128, 128), 6)]


@pytest.mark.parametrize("shape,n_tc", TC_SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}" for s, _ in TC_SHAPES])
def test_tensor_memory_forward_matches_oracle(shape, n_tc):
    """tcgen05 convolutions (FP32 accumulators in tensor memory) against the oracle with
    the GPU's BF16 storage emulated: the remaining differences are FP32 summation
    order and the BF16 roundings it flips (bound 5e-3 normwise); against the plain FP64
    oracle 2e-2 as for the mma.sync kernel.  The mma.sync kernel on the same network and
    input agrees to 5e-3."""
    net, x, params = make(1, *shape)
    info = net.kernel_info()
    assert info["tc_forward"] == n_tc and info["fault"] == 0, info
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    y = net.forward(xt).cpu().numpy().reshape(shape)
    assert net.kernel_info()["fault"] == 0
    y_bf = forward_bf16_storage(params, x)
    y_or, _ = onn.forward(params, x)
    net.use_tensor_memory(False)
    assert net.kernel_info()["tc_forward"] == 0
    y_ms = net.forward(xt).cpu().numpy().reshape(shape)
    print(f"{shape}: rel err vs BF16-storage oracle {rel(y, y_bf):.2e}, vs FP64 oracle {rel(y, y_or):.2e}, "
          f"vs mma.sync {rel(y, y_ms):.2e}")
    assert rel(y, y_bf) <= 5e-3
    assert rel(y, y_or) <= 2e-2
    assert rel(y, y_ms) <= 5e-3
    net.close()


def test_tensor_memory_gradients_match_oracle():
    """Backward pass with the adjoint convolutions on the tcgen05 kernel (all five at
    4x32x16) against the oracle with BF16 storage emulated, as for the mma.sync path."""
    net, x, params = make(2, 4, 32, 16)
    assert net.kernel_info()["tc_backward"] == 5
    t = np.random.default_rng(3).standard_normal((4, 32, 16))
    loss_or, g_or = forward_backward_bf16_storage(params, x, t)
    xt = torch.as_tensor(x.reshape(-1, 16), dtype=torch.float32, device="cuda")
    tt = torch.as_tensor(t.ravel(), dtype=torch.float32, device="cuda")
    loss = net.loss_grad(xt, tt)
    _, _, gw, gb = net.params()
    assert net.kernel_info()["fault"] == 0
    assert abs(loss - loss_or) <= 2e-2 * loss_or
    for layer in range(6):
        e_w = rel(gw[layer], g_or[layer][0].reshape(27, *g_or[layer][0].shape[3:]))
        e_b = rel(gb[layer], g_or[layer][1])
        print(f"layer {layer}: grad rel err w {e_w:.2e} b {e_b:.2e}")
        assert e_w <= 2e-2 and e_b <= 2e-2, (layer, e_w, e_b)
    net.close()


def test_use_tensor_memory_rejects_other_values():
    from paper_2210_15668_gb300 import ferrox
    net, _, _ = make(1, 4, 16, 8)
    with pytest.raises(ferrox.FerroxError, match="EINVAL"):
        net._ck(net.lib.ferrox_nn_use_tensor_memory(net.ctx, 2))
    net.close()
