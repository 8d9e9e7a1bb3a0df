"""Pins of the FP64 denoiser oracle: the convolution against scipy's
correlate, its gradients through the adjoint identities and finite
differences, and the whole U-Net backward pass by finite differences."""
import numpy as np
import pytest
from scipy import ndimage


@pytest.fixture(scope="module")
def dn():
    from oracle import denoise
    return denoise


def test_conv3d_matches_scipy_correlate(dn):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5, 2))
    w = rng.normal(size=(3, 27, 2))
    b = rng.normal(size=3)
    y = dn.conv3d(x, w, b)
    for n in range(2):
        for co in range(3):
            ref = b[co] + sum(ndimage.correlate(x[n, ..., ci], w[co, :, ci].reshape(3, 3, 3), mode="constant", cval=0.0)
                              for ci in range(2))
            assert np.allclose(y[n, ..., co], ref, atol=1e-12)


def test_conv3d_gradients_are_adjoints(dn):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 4, 3, 5, 3))
    w = rng.normal(size=(2, 27, 3))
    g = rng.normal(size=(1, 4, 3, 5, 2))
    lhs = np.sum(dn.conv3d(x, w) * g)
    assert abs(lhs - np.sum(x * dn.conv3d_dgrad(g, w))) < 1e-10 * abs(lhs) + 1e-10
    dw, db = dn.conv3d_wgrad(x, g)
    assert abs(lhs - np.sum(w * dw)) < 1e-10 * abs(lhs) + 1e-10
    assert np.allclose(db, g.reshape(-1, 2).sum(0))
    # finite differences on a few weights
    for (co, t, ci) in [(0, 0, 0), (1, 13, 2), (0, 26, 1)]:
        e = 1e-6
        wp = w.copy(); wp[co, t, ci] += e
        wm = w.copy(); wm[co, t, ci] -= e
        fd = (np.sum(dn.conv3d(x, wp) * g) - np.sum(dn.conv3d(x, wm) * g)) / (2 * e)
        assert abs(fd - dw[co, t, ci]) < 1e-6 * max(1, abs(fd))


def test_pool_and_upsample_adjoints(dn):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 6, 2, 3))
    g = rng.normal(size=(1, 2, 3, 1, 3))
    assert abs(np.sum(dn.avgpool2(x) * g) - np.sum(x * dn.avgpool2_adjoint(g))) < 1e-12
    assert abs(np.sum(dn.upsample2(g) * x) - np.sum(g * dn.upsample2_adjoint(x))) < 1e-12
    assert np.allclose(dn.avgpool2(np.ones((1, 2, 2, 2, 1))), 1.0)


def test_unet_backward_matches_finite_differences(dn):
    rng = np.random.default_rng(3)
    widths = (4, 8, 8)
    x = rng.normal(size=(1, 8, 8, 8, 3))
    params = dn.unet_init(rng, cin=3, widths=widths, scale=1.5)
    gy = rng.normal(size=(1, 8, 8, 8))
    y, cache = dn.unet_forward(x, params, widths)
    grads = dn.unet_backward(gy, params, cache, widths)
    loss = lambda p: np.sum(dn.unet_forward(x, p, widths)[0] * gy)
    names = [n for n, _, _ in dn.unet_layers(3, widths)] + ["head"]
    assert set(grads) == set(names)
    checked = 0
    for name in names:
        w, b = params[name]
        gw, gb = grads[name]
        idx = tuple(int(rng.integers(0, s)) for s in w.shape)
        for which in ("w", "b"):
            e = 1e-6
            p_plus = dict(params); p_minus = dict(params)
            if which == "w":
                wp = w.copy(); wp[idx] += e; wm = w.copy(); wm[idx] -= e
                p_plus[name] = (wp, b); p_minus[name] = (wm, b)
                an = gw[idx]
            else:
                j = int(rng.integers(0, b.shape[0]))
                bp = b.copy(); bp[j] += e; bm = b.copy(); bm[j] -= e
                p_plus[name] = (w, bp); p_minus[name] = (w, bm)
                an = gb[j]
            fd = (loss(p_plus) - loss(p_minus)) / (2 * e)
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (name, which, fd, an)
            checked += 1
    assert checked == 2 * len(names)


def test_adam_two_steps_by_hand():
    # w0 = 1, gradients 0.5 then -0.25, lr 0.1, beta1 0.9, beta2 0.999, eps 1e-8.
    # Step 1: m = 0.1*0.5 = 0.05, v = 0.001*0.25 = 0.00025; corrected 0.5 and
    #   0.25; w = 1 - 0.1*0.5/(0.5 + 1e-8) = 0.90000000199999996...
    # Step 2: m = 0.9*0.05 - 0.1*0.25 = 0.02, v = 0.999*0.00025 + 0.001*0.0625
    #   = 0.00031225; corrected 0.02/0.19 and 0.00031225/0.001999;
    #   w = 0.9000000019999... - 0.1*0.105263157894737/(0.395225379... + 1e-8)
    #     = 0.87336629870784616...  (40-digit decimal arithmetic)
    from oracle import denoise as dn
    w, m, v = dn.adam_step(np.array([1.0]), np.array([0.5]), 0.0, 0.0, 1, 0.1)
    # (1 - 0.9 is 0.09999999999999998 in FP64: relative 1e-14 covers the rounding)
    assert abs(m[0] / 0.05 - 1) < 1e-14 and abs(v[0] / 0.00025 - 1) < 1e-14
    assert abs(w[0] - 0.90000000199999996) < 1e-15
    w, m, v = dn.adam_step(w, np.array([-0.25]), m, v, 2, 0.1)
    assert abs(m[0] / 0.02 - 1) < 1e-14 and abs(v[0] / 0.00031225 - 1) < 1e-14
    assert abs(w[0] - 0.87336629870784616) < 1e-15


def test_adam_first_step_moves_every_weight_by_lr():
    # At t = 1 the corrected moments are g and g^2, so each weight moves by
    # lr g / (|g| + eps): lr against the gradient's sign, whatever its size.
    from oracle import denoise as dn
    rng = np.random.default_rng(0)
    g = rng.normal(size=1000) * 10.0 ** rng.uniform(-3, 3, 1000)
    w0 = rng.normal(size=1000)
    w, _, _ = dn.adam_step(w0, g, 0.0, 0.0, 1, 1e-3, eps=0.0)
    assert np.allclose(w0 - w, 1e-3 * np.sign(g), rtol=1e-12, atol=0)
