"""The GPU U-Net (forward, backward, Adam, whole-volume apply) against the FP64
oracle U-Net on the same BF16-rounded weights and inputs.

The GPU keeps every activation and activation gradient in BF16 (relative
rounding 2^-9 per layer), so outputs and gradients agree with the FP64 oracle
to about a percent, not bitwise; the tolerances below are stated per check."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from oracle import denoise
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return torch, nmdose, denoise


def to_oracle(flat, layers, widths, names):
    params = {}
    for name, l in zip(names, layers[:-1]):
        w = flat[l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])[:, :27 * l["cin"]]
        params[name] = (w.reshape(l["cout"], 27, l["cin"]).astype(np.float64),
                        flat[l["b_off"]:l["b_off"] + l["cout"]].astype(np.float64))
    h = layers[-1]
    params["head"] = (flat[h["w_off"]:h["w_off"] + widths[0]][None, :].astype(np.float64),
                      flat[h["b_off"]:h["b_off"] + 1].astype(np.float64))
    return params


def grads_from_flat(flat, layers, names, widths):
    return to_oracle(flat, layers, widths, names)


def bf16_round(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def test_unet_matches_oracle_forward_and_gradients(env):
    torch, nm, dn = env
    P, widths = 16, (16, 32, 64, 128)
    net = nm.Denoiser(patch=P, batch=1, levels=4, base_width=16, seed=3)
    layers = net.layers()
    names = [n for n, _, _ in dn.unet_layers(8, widths)]
    assert len(layers) == len(names) + 1
    rng = np.random.default_rng(5)
    flat = np.zeros(net.n_params, np.float32)
    net.params(get=flat)
    # bias and head away from zero so that every path carries gradient
    for l in layers[:-1]:
        flat[l["b_off"]:l["b_off"] + l["cout"]] = rng.normal(0, 0.05, l["cout"])
        w = flat[l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])
        w[:, :27 * l["cin"]] = bf16_round(torch, w[:, :27 * l["cin"]])   # exact in BF16
    h = layers[-1]
    flat[h["w_off"]:h["w_off"] + widths[0]] = rng.normal(0, 0.3, widths[0])
    flat[h["b_off"]] = 0.1
    net.params(set=flat)
    x = np.zeros((1, P, P, P, 8), np.float32)
    x[..., :3] = rng.normal(0, 1, (1, P, P, P, 3))
    xb = torch.from_numpy(x).to(torch.bfloat16)
    x64 = xb.float().numpy().astype(np.float64)
    target = rng.normal(0, 1, (1, P, P, P)).astype(np.float32)
    weight = (rng.random((1, P, P, P)) < 0.7).astype(np.float32)
    loss = net.train_step(xb.cuda(), torch.from_numpy(target).cuda(), torch.from_numpy(weight).cuda(), lr=0.0)
    g = np.zeros(net.n_params, np.float32)
    net.params(grads=g)
    y = torch.empty((1, P, P, P), dtype=torch.float32, device="cuda")
    net.forward(xb.cuda(), y)
    y = y.cpu().numpy()
    params = to_oracle(flat, layers, widths, names)
    yo, cache = dn.unet_forward(x64, params, widths)
    m = yo.size
    assert np.linalg.norm(y - yo) / np.linalg.norm(yo) < 2e-2
    lo = np.sum(weight * (yo - target) ** 2) / m
    assert abs(loss / lo - 1) < 3e-2, (loss, lo)
    go = dn.unet_backward(2 * weight * (yo - target) / m, params, cache, widths)
    gg = grads_from_flat(g, layers, names, widths)
    for name in names + ["head"]:
        for k in range(2):
            a, b = gg[name][k].ravel(), go[name][k].ravel()
            rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
            # BF16 activations and gradients at ~10 stages between the loss and the
            # deepest layers, plus ReLU masks that flip where a pre-activation is
            # within rounding of zero: direction within 8 degrees, norm within 15 %.
            assert rel < 0.15 and cos > 0.99, (name, k, rel, cos)
    # padding columns of every weight matrix get exactly zero gradient
    for l in layers[:-1]:
        gw = g[l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])
        assert np.all(gw[:, 27 * l["cin"]:] == 0.0)
    net.close()


def test_unet_training_reduces_loss(env):
    torch, nm, dn = env
    P, B = 32, 2
    net = nm.Denoiser(patch=P, batch=B, levels=4, base_width=16, seed=1, lr=2e-3)
    rng = np.random.default_rng(0)
    zz, yy, xx = np.meshgrid(*[np.arange(P)] * 3, indexing="ij")
    losses = []
    for step in range(80):
        clean = np.zeros((B, P, P, P), np.float32)
        x = np.zeros((B, P, P, P, 8), np.float32)
        for b in range(B):
            c = rng.uniform(8, 24, 3)
            r = rng.uniform(4, 10)
            clean[b] = 2.0 * np.exp(-((zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2) / (2 * r * r))
            x[b, ..., 0] = clean[b] + rng.normal(0, 0.3, (P, P, P))
            x[b, ..., 1] = 1.0
        loss = net.train_step(torch.from_numpy(x).to(torch.bfloat16).cuda(), torch.from_numpy(clean).cuda())
        losses.append(loss)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5]), (losses[:5], losses[-10:])
    net.close()


def test_apply_covers_the_volume(env):
    torch, nm, dn = env
    # A fresh network's head is zero: it returns its input dose channel, so a
    # whole-volume apply must give back the input (to BF16 precision) in every voxel.
    net = nm.Denoiser(patch=32, batch=3, levels=4, base_width=16, seed=2)
    rng = np.random.default_rng(1)
    shape = (40, 48, 56)
    dose = rng.lognormal(-15, 0.5, shape).astype(np.float32)
    den = np.where(rng.random(shape) < 0.8, 1.0, 0.001).astype(np.float32)
    act = rng.lognormal(0, 0.3, shape).astype(np.float32)
    out = torch.full(shape, -1.0, dtype=torch.float32, device="cuda")
    net.apply(torch.from_numpy(dose).cuda(), torch.from_numpy(den).cuda(), torch.from_numpy(act).cuda(), out)
    o = out.cpu().numpy()
    assert np.all(o > 0)
    assert np.allclose(o, dose, rtol=1e-2)
    net.close()
