"""Oracle of the learned preconditioner: the 3-level 3-D encoder-decoder in plain FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see oracle/poisson.py): only tests/ import it.  It shares no code with
the CUDA library.  A convolution is written out from its definition, a sum over the 27 taps of a
shifted input times that tap's weight matrix (numpy matmul as the step); pooling is the mean of
each 2x2x2 block and upsampling copies a coarse cell to its 8 children.  Backward passes are the
transposes of those definitions.  With ``bf16=True`` every value that the GPU stores in BF16 is
rounded to BF16 (round to nearest even) at the same point, so the two agree to BF16 accuracy;
with ``bf16=False`` the computation is pure FP64 (used for the finite-difference check).

Tensors are channels-last, shape (nz, ny, nx, C).  Weights of a layer: W[27][cout][cin] with tap
index (dz+1)*9 + (dy+1)*3 + (dx+1); parameters are flattened layer by layer (weights, then bias),
then the output layer's 16 weights and its bias.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), via FP32 like the GPU's conversions."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    layers, off = [], 0
    for cin, cout in LAYERS:
        n = 27 * cout * cin
        W = flat[off:off + n].reshape(27, cout, cin)
        off += n
        b = flat[off:off + cout]
        off += cout
        layers.append((W, b))
    hw = flat[off:off + 16]
    hb = flat[off + 16]
    assert off + 17 == flat.size
    return layers, hw, hb


def pack(layers, hw, hb):
    parts = []
    for W, b in layers:
        parts += [W.ravel(), b.ravel()]
    parts += [np.asarray(hw).ravel(), np.array([hb])]
    return np.concatenate(parts)


def _shift_view(xp, tap, shape):
    nz, ny, nx = shape
    dz, dy, dx = tap // 9, (tap // 3) % 3, tap % 3
    return xp[dz:dz + nz, dy:dy + ny, dx:dx + nx, :]


def conv3(x, W, b):
    """out[v, co] = b[co] + sum over taps and ci of x[v + tap - 1, ci] W[tap, co, ci] (zero padding)."""
    shape = x.shape[:3]
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros(shape + (W.shape[1],))
    for tap in range(27):
        out += _shift_view(xp, tap, shape) @ W[tap].T
    if b is not None:
        out += b
    return out


def conv3_data_grad(dy, W, shape):
    """dx[u, ci] = sum over taps and co of dy[u - tap + 1, co] W[tap, co, ci]."""
    dxp = np.zeros((shape[0] + 2, shape[1] + 2, shape[2] + 2, W.shape[2]))
    for tap in range(27):
        dz, dyy, dx = tap // 9, (tap // 3) % 3, tap % 3
        dxp[dz:dz + shape[0], dyy:dyy + shape[1], dx:dx + shape[2], :] += dy @ W[tap]
    return dxp[1:-1, 1:-1, 1:-1, :]


def conv3_weight_grad(x, dy):
    """dW[tap, co, ci] = sum over voxels v of dy[v, co] x[v + tap - 1, ci]."""
    shape = x.shape[:3]
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    V = int(np.prod(shape))
    d2 = dy.reshape(V, -1)
    return np.stack([d2.T @ _shift_view(xp, tap, shape).reshape(V, -1) for tap in range(27)])


def pool(x):
    nz, ny, nx, C = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, C).mean(axis=(1, 3, 5))


def pool_grad(d):
    return np.repeat(np.repeat(np.repeat(d, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_grad(d):
    nz, ny, nx, C = d.shape
    return d.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, C).sum(axis=(1, 3, 5))


def geometry(F, apertures, dx, dy, dz):
    """Seven input channels per cell: F, the mean open fraction of the cell's two x, y and z faces,
    log(dx/dx_min), log(dy/dy_min), log(dz/dz_min)."""
    ex, ey, ez = apertures
    nz, ny, nx = F.shape
    g = np.zeros((nz, ny, nx, 8))
    g[..., 0] = F
    g[..., 1] = 0.5 * (ex[:, :, :-1] + ex[:, :, 1:])
    g[..., 2] = 0.5 * (ey[:, :-1, :] + ey[:, 1:, :])
    g[..., 3] = 0.5 * (ez[:-1] + ez[1:])
    g[..., 4] = np.log(dx / dx.min())[None, None, :]
    g[..., 5] = np.log(dy / dy.min())[None, :, None]
    g[..., 6] = np.log(dz / dz.min())[:, None, None]
    return g


def forward(params, geo, mask, r, bf16=True):
    """Network output z (nz, ny, nx) for the scaled residual r; returns (z, cache)."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers, hw, hb = unpack(params)
    Wr = [(rnd(W), b) for W, b in layers]
    rms = np.sqrt((mask * r * r).sum() / mask.sum())
    inv = 1.0 / rms
    x0 = np.zeros(r.shape + (16,))
    x0[..., :7] = rnd(geo[..., :7])
    x0[..., 7] = rnd(r * inv)
    relu = lambda a: np.maximum(a, 0.0)
    c = {"x0": x0, "rms": rms, "mask": mask}
    c["a1"] = rnd(relu(conv3(x0, *Wr[0])))
    c["s1"] = rnd(relu(conv3(c["a1"], *Wr[1])))
    c["p1"] = rnd(pool(c["s1"]))
    c["a2"] = rnd(relu(conv3(c["p1"], *Wr[2])))
    c["s2"] = rnd(relu(conv3(c["a2"], *Wr[3])))
    c["p2"] = rnd(pool(c["s2"]))
    c["a3"] = rnd(relu(conv3(c["p2"], *Wr[4])))
    c["b3"] = rnd(relu(conv3(c["a3"], *Wr[5])))
    c["c2"] = np.concatenate([up(c["b3"]), c["s2"]], axis=-1)
    c["d2a"] = rnd(relu(conv3(c["c2"], *Wr[6])))
    c["d2b"] = rnd(relu(conv3(c["d2a"], *Wr[7])))
    c["c1"] = np.concatenate([up(c["d2b"]), c["s1"]], axis=-1)
    c["d1a"] = rnd(relu(conv3(c["c1"], *Wr[8])))
    c["d1b"] = rnd(relu(conv3(c["d1a"], *Wr[9])))
    z = mask * (c["d1b"] @ hw + hb) * rms
    c["Wr"] = Wr
    c["hw"] = hw
    return z, c


def loss_and_grads(params, geo, mask, r, target, bf16=True):
    """Masked mean-squared error of (z - target)/rms over cells with an unknown, and its gradient
    with respect to every parameter (flattened like the parameters)."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    z, c = forward(params, geo, mask, r, bf16)
    count = mask.sum()
    e = mask * (z - target) / c["rms"]
    loss = (e * e).sum() / count
    go = 2.0 * e / count
    hw = c["hw"]
    g_hw = np.einsum("zyx,zyxc->c", go, c["d1b"])
    g_hb = go.sum()
    grads = [None] * 10
    Wr = c["Wr"]

    def layer(i, x, y, dy, want_dx):
        dpre = dy * (y > 0)
        grads[i] = (conv3_weight_grad(x, dpre), dpre.sum(axis=(0, 1, 2)))
        return rnd(conv3_data_grad(dpre, Wr[i][0], x.shape[:3])) if want_dx else None

    d = rnd(go[..., None] * hw)
    d = layer(9, c["d1a"], c["d1b"], d, True)
    d = layer(8, c["c1"], c["d1a"], d, True)
    g_d2b = rnd(up_grad(d[..., :32]))
    g_s1 = rnd(d[..., 32:])
    d = layer(7, c["d2a"], c["d2b"], g_d2b, True)
    d = layer(6, c["c2"], c["d2a"], d, True)
    g_b3 = rnd(up_grad(d[..., :64]))
    g_s2 = rnd(d[..., 64:])
    d = layer(5, c["a3"], c["b3"], g_b3, True)
    g_p2 = layer(4, c["p2"], c["a3"], d, True)
    g_s2 = rnd(g_s2 + pool_grad(g_p2))
    d = layer(3, c["a2"], c["s2"], g_s2, True)
    g_p1 = layer(2, c["p1"], c["a2"], d, True)
    g_s1 = rnd(g_s1 + pool_grad(g_p1))
    d = layer(1, c["a1"], c["s1"], g_s1, True)
    layer(0, c["x0"], c["a1"], d, False)
    return loss, pack([g for g in grads], g_hw, g_hb), z


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) with the bias-corrected step size."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    lr_t = lr * np.sqrt(1 - b2 ** step) / (1 - b1 ** step)
    return params - lr_t * m / (np.sqrt(v) + eps), m, v
