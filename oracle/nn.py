"""FP64 reference of the learned warm-start network (oracle; test infrastructure).

The network is not in the paper (the workloads add it): a small two-resolution
3-D U-Net that maps features of the initial residual of a Poisson solve, on a
coarse multigrid level, to the error of the initial guess on that level.
Channels-last arrays [D][H][W][C] (z, y, x, channel).  Convolutions are 3x3x3,
periodic in x and y (the device is periodic laterally) and zero-padded in z
(electrodes).  Pooling is the 2x2x2 mean; upsampling repeats each coarse value
over its 2x2x2 children.

    x (CIN) -> conv(CIN,16) relu -> conv(16,16) relu = s1
            -> pool -> conv(16,32) relu -> conv(32,32) relu
            -> up -> concat(., s1) (48) -> conv(48,16) relu -> conv(16,16) -> out[..., 0]

Each layer's weights are [3][3][3][Cin][Cout] and a bias [Cout].  The GPU path
stores weights and activations in BF16 and accumulates in FP32; this reference
takes the same (BF16-rounded) numbers in FP64.
"""
import numpy as np

CIN = 16          # input channels (features are zero-padded to 16)
LAYERS = [(CIN, 16), (16, 16), (16, 32), (32, 32), (48, 16), (16, 16)]
RELU = [True, True, True, True, True, False]


def conv3d(x, w, b):
    """out[z,y,x,co] = b[co] + sum_{dz,dy,dx,ci} x[z+dz-1, y+dy-1, x+dx-1, ci] w[dz,dy,dx,ci,co]."""
    D, H, W, _ = x.shape
    xp = np.zeros((D + 2, H, W, x.shape[3]))
    xp[1:-1] = x
    out = np.broadcast_to(b, (D, H, W, w.shape[4])).astype(np.float64).copy()
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sh = np.roll(np.roll(xp[dz:dz + D], 1 - dy, axis=1), 1 - dx, axis=2)
                out += np.tensordot(sh, w[dz, dy, dx], axes=([3], [0]))
    return out


def conv3d_backward(x, w, dout):
    """(dx, dw, db) of conv3d for the upstream gradient dout."""
    D, H, W, _ = x.shape
    xp = np.zeros((D + 2, H, W, x.shape[3]))
    xp[1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sh = np.roll(np.roll(xp[dz:dz + D], 1 - dy, axis=1), 1 - dx, axis=2)
                dw[dz, dy, dx] = np.tensordot(sh, dout, axes=([0, 1, 2], [0, 1, 2]))
                g = np.tensordot(dout, w[dz, dy, dx], axes=([3], [1]))
                dxp[dz:dz + D] += np.roll(np.roll(g, dy - 1, axis=1), dx - 1, axis=2)
    return dxp[1:-1], dw, dout.sum(axis=(0, 1, 2))


def pool2(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool2_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 0), 2, 1), 2, 2) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up2_backward(dy):
    D, H, W, C = dy.shape
    return dy.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def forward(params, x):
    """params: list of (w, b); returns (output channel 0, cache)."""
    a1 = np.maximum(conv3d(x, *params[0]), 0.0)
    s1 = np.maximum(conv3d(a1, *params[1]), 0.0)
    p = pool2(s1)
    a3 = np.maximum(conv3d(p, *params[2]), 0.0)
    a4 = np.maximum(conv3d(a3, *params[3]), 0.0)
    cat = np.concatenate([up2(a4), s1], axis=3)
    a5 = np.maximum(conv3d(cat, *params[4]), 0.0)
    y = conv3d(a5, *params[5])
    cache = (x, a1, s1, p, a3, a4, cat, a5)
    return y[..., 0], cache


def backward(params, cache, dy0):
    """Gradients (list of (dw, db)) for d(loss)/d(output channel 0) = dy0."""
    x, a1, s1, p, a3, a4, cat, a5 = cache
    dy = np.zeros(dy0.shape + (params[5][0].shape[4],))
    dy[..., 0] = dy0
    g = [None] * 6
    da5, *g5 = conv3d_backward(a5, params[5][0], dy)
    g[5] = tuple(g5)
    da5 = da5 * (a5 > 0)
    dcat, *g4 = conv3d_backward(cat, params[4][0], da5)
    g[4] = tuple(g4)
    da4 = up2_backward(dcat[..., :32]) * (a4 > 0)
    ds1 = dcat[..., 32:]
    da3, *g3 = conv3d_backward(a3, params[3][0], da4)
    g[3] = tuple(g3)
    da3 = da3 * (a3 > 0)
    dp, *g2 = conv3d_backward(p, params[2][0], da3)
    g[2] = tuple(g2)
    ds1 = (ds1 + pool2_backward(dp)) * (s1 > 0)
    da1, *g1 = conv3d_backward(a1, params[1][0], ds1)
    g[1] = tuple(g1)
    da1 = da1 * (a1 > 0)
    _, *g0 = conv3d_backward(x, params[0][0], da1)
    g[0] = tuple(g0)
    return g


def mse(y, t):
    """Mean squared error and its gradient with respect to y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of every weight and bias, in place."""
    out = []
    for q, ((w, b), (dw, db)) in enumerate(zip(params, grads)):
        new = []
        for r, (p_, g_) in enumerate(((w, dw), (b, db))):
            m[q][r] = beta1 * m[q][r] + (1 - beta1) * g_
            v[q][r] = beta2 * v[q][r] + (1 - beta2) * g_ * g_
            mh = m[q][r] / (1 - beta1 ** step)
            vh = v[q][r] / (1 - beta2 ** step)
            new.append(p_ - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out
