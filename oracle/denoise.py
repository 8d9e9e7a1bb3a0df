"""FP64 reference of the dose denoiser: 3x3x3 convolutions (forward, input and
weight gradients) and the 3D U-Net built from them, with its backward pass.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The denoiser is not in
the paper; these definitions are the plain textbook ones: a convolution is a
sum over the 27 taps of a shifted copy of the input times that tap's weight
matrix, zero outside the volume, and its gradients are the adjoints of that
sum.  Arrays are channels-last [n, d, h, w, c] in float64; weights are
[cout, 27, cin] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(xp, t, shape):
    dz, dy, dx = TAPS[t]
    _, d, h, w, _ = shape
    return xp[:, 1 + dz:1 + dz + d, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w, :]


def conv3d(x, w, b=None):
    """y[p, co] = sum_t sum_ci x[p + off_t, ci] w[co, t, ci] (+ b[co])."""
    x = np.asarray(x, np.float64)
    n, d, h, ww, cin = x.shape
    cout = w.shape[0]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((n, d, h, ww, cout))
    for t in range(27):
        y += _shift(xp, t, x.shape) @ w[:, t, :].T
    if b is not None:
        y += b
    return y


def conv3d_dgrad(dy, w):
    """Adjoint of conv3d in x: dx[q] = sum_t dy[q - off_t] w[:, t, :]."""
    dy = np.asarray(dy, np.float64)
    n, d, h, ww, _ = dy.shape
    cin = w.shape[2]
    dxp = np.zeros((n, d + 2, h + 2, ww + 2, cin))
    for t, (dz, dyy, dx) in enumerate(TAPS):
        dxp[:, 1 + dz:1 + dz + d, 1 + dyy:1 + dyy + h, 1 + dx:1 + dx + ww, :] += dy @ w[:, t, :]
    return dxp[:, 1:-1, 1:-1, 1:-1, :]


def conv3d_wgrad(x, dy):
    """Adjoint of conv3d in w: dw[co, t, ci] = sum_p dy[p, co] x[p + off_t, ci]; db = sum_p dy."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    cin = x.shape[4]
    cout = dy.shape[4]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((cout, 27, cin))
    dyf = dy.reshape(-1, cout)
    for t in range(27):
        dw[:, t, :] = dyf.T @ _shift(xp, t, x.shape).reshape(-1, cin)
    return dw, dyf.sum(axis=0)


def upsample2(x):
    """Nearest-neighbour upsampling by 2 in each spatial axis."""
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_adjoint(g):
    n, d, h, w, c = g.shape
    return g.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4, 6))


def avgpool2(x):
    n, d, h, w, c = x.shape
    return x.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4, 6))


def avgpool2_adjoint(g):
    return upsample2(g) / 8.0


# ---------------------------------------------------------------------------
# The U-Net: 4 levels with widths (16, 32, 64, 128) by default, two 3x3x3
# convolutions with ReLU per level, average pooling down, nearest upsampling
# and concatenation with the skip connection up, a 1x1x1 head.  The output is
# added to input channel 0 (a residual on the log-normalised low-count dose).
# ---------------------------------------------------------------------------
def unet_layers(cin=8, widths=(16, 32, 64, 128)):
    """(name, cin_total, cout) of every 3x3x3 convolution, in forward order."""
    L = []
    c = cin
    for i, wd in enumerate(widths):
        L.append((f"e{i}a", c, wd))
        L.append((f"e{i}b", wd, wd))
        c = wd
    for i in range(len(widths) - 2, -1, -1):
        L.append((f"d{i}a", c + widths[i], widths[i]))
        L.append((f"d{i}b", widths[i], widths[i]))
        c = widths[i]
    return L


def unet_forward(x, params, widths=(16, 32, 64, 128)):
    """x [n,d,h,w,cin]; params: {name: (w [cout,27,cin], b [cout])} plus
    'head': (w [1, cout0], b [1]).  Returns (y [n,d,h,w], cache)."""
    cache = {"x": x}
    h = x
    skips = []
    nl = len(widths)
    for i in range(nl):
        wa, ba = params[f"e{i}a"]
        a = np.maximum(conv3d(h, wa, ba), 0.0)
        wb, bb = params[f"e{i}b"]
        o = np.maximum(conv3d(a, wb, bb), 0.0)
        cache[f"e{i}a_in"], cache[f"e{i}a_out"] = h, a
        cache[f"e{i}b_out"] = o
        skips.append(o)
        h = avgpool2(o) if i < nl - 1 else o
    for i in range(nl - 2, -1, -1):
        cat = np.concatenate([upsample2(h), skips[i]], axis=4)
        wa, ba = params[f"d{i}a"]
        a = np.maximum(conv3d(cat, wa, ba), 0.0)
        wb, bb = params[f"d{i}b"]
        o = np.maximum(conv3d(a, wb, bb), 0.0)
        cache[f"d{i}a_in"], cache[f"d{i}a_out"], cache[f"d{i}b_out"] = cat, a, o
        h = o
    hw, hb = params["head"]
    y = h @ hw[0] + hb[0] + x[..., 0]
    cache["top"] = h
    return y, cache


def unet_backward(gy, params, cache, widths=(16, 32, 64, 128)):
    """Gradients of sum(gy * y) with respect to every parameter."""
    grads = {}
    nl = len(widths)
    hw, hb = params["head"]
    top = cache["top"]
    grads["head"] = ((gy[..., None] * top).reshape(-1, top.shape[-1]).sum(0)[None, :],
                     np.array([gy.sum()]))
    g = gy[..., None] * hw[0]                      # d top
    skip_grads = [None] * nl
    # decoder, in reverse forward order: i = 0 .. nl-2
    for i in range(0, nl - 1):
        o = cache[f"d{i}b_out"]
        g = g * (o > 0)
        wb, _ = params[f"d{i}b"]
        grads[f"d{i}b"] = conv3d_wgrad(cache[f"d{i}a_out"], g)
        g = conv3d_dgrad(g, wb) * (cache[f"d{i}a_out"] > 0)
        wa, _ = params[f"d{i}a"]
        grads[f"d{i}a"] = conv3d_wgrad(cache[f"d{i}a_in"], g)
        gc = conv3d_dgrad(g, wa)
        cu = gc.shape[-1] - widths[i]
        skip_grads[i] = gc[..., cu:]
        g = upsample2_adjoint(gc[..., :cu])          # gradient of the coarser level's output
    # encoder, deepest first
    for i in range(nl - 1, -1, -1):
        o = cache[f"e{i}b_out"]
        if i < nl - 1:
            g = avgpool2_adjoint(g) + skip_grads[i]
        g = g * (o > 0)
        wb, _ = params[f"e{i}b"]
        grads[f"e{i}b"] = conv3d_wgrad(cache[f"e{i}a_out"], g)
        g = conv3d_dgrad(g, wb) * (cache[f"e{i}a_out"] > 0)
        wa, _ = params[f"e{i}a"]
        grads[f"e{i}a"] = conv3d_wgrad(cache[f"e{i}a_in"], g)
        if i > 0:
            g = conv3d_dgrad(g, wa)
    return grads


def unet_init(rng, cin=8, widths=(16, 32, 64, 128), scale=1.0):
    params = {}
    for name, ci, co in unet_layers(cin, widths):
        std = scale * np.sqrt(2.0 / (27 * ci))
        params[name] = (rng.normal(0, std, (co, 27, ci)), rng.normal(0, 0.01, co))
    params["head"] = (rng.normal(0, np.sqrt(1.0 / widths[0]), (1, widths[0])), np.zeros(1))
    return params


def adam_step(w, g, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) in FP64: the biased
    first and second moment estimates, their bias corrections at update t
    (counted from 1), and the parameter step.  Returns new (w, m1, m2)."""
    w, g = np.asarray(w, np.float64), np.asarray(g, np.float64)
    m1 = beta1 * np.asarray(m1, np.float64) + (1.0 - beta1) * g
    m2 = beta2 * np.asarray(m2, np.float64) + (1.0 - beta2) * g * g
    m_hat = m1 / (1.0 - beta1 ** t)
    v_hat = m2 / (1.0 - beta2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m1, m2
