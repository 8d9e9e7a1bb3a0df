"""The GPU U-Net checked layer by layer and element by element against the FP64
oracle, each check fed the GPU's own BF16 tensors so that rounding does not
accumulate across layers: every convolution's forward output, weight and
bias gradients, every kernel between convolutions (pooling, upsampling and
concatenation, the split of a decoder input's gradient, the encoder's
gradient sum, the ReLU masks, the head), and two Adam updates (master
weights and both moments).

Tolerances come from the arithmetic: a BF16 result carries a rounding of at
most 2^-8 of its magnitude (8 significant bits) per rounding it went
through, an FP32 sum of K terms at most about K 2^-24 of the sum of their
magnitudes."""
import numpy as np
import pytest

from tests.parity_record import record

pytestmark = pytest.mark.gpu

P, WIDTHS = 16, (16, 32, 64, 128)
U8 = 2.0 ** -8


@pytest.fixture(scope="module")
def run():
    """One captured training step (lr = 0) of a 4-level U-Net on a 16^3 patch,
    then two Adam steps, with everything the checks need on the host."""
    import torch

    from oracle import denoise as dn
    from paper_2111_11687_gb300 import build, nmdose as nm
    build.build()
    nm.load()
    net = nm.Denoiser(patch=P, batch=1, levels=4, base_width=16, seed=3, lr=1e-3)
    layers = net.layers()
    names = [n for n, _, _ in dn.unet_layers(8, WIDTHS)]
    rng = np.random.default_rng(7)
    flat = np.zeros(net.n_params, np.float32)
    net.params(get=flat)
    for l in layers[:-1]:
        flat[l["b_off"]:l["b_off"] + l["cout"]] = rng.normal(0, 0.05, l["cout"])
        w = flat[l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])
        w[:, :27 * l["cin"]] = torch.from_numpy(np.ascontiguousarray(w[:, :27 * l["cin"]])).to(
            torch.bfloat16).float().numpy()                      # exactly representable in BF16
    h = layers[-1]
    flat[h["w_off"]:h["w_off"] + WIDTHS[0]] = rng.normal(0, 0.3, WIDTHS[0])
    flat[h["b_off"]] = 0.1
    net.params(set=flat)
    x = np.zeros((1, P, P, P, 8), np.float32)
    x[..., :4] = rng.normal(0, 1, (1, P, P, P, 4))
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    target = torch.from_numpy(rng.normal(0, 1, (1, P, P, P)).astype(np.float32)).cuda()
    weight = torch.from_numpy((rng.random((1, P, P, P)) < 0.7).astype(np.float32)).cuda()
    net.capture(True)
    loss = net.train_step(xb, target, weight, lr=0.0)
    g0 = np.zeros(net.n_params, np.float32)
    net.params(grads=g0)
    y = torch.empty((1, P, P, P), dtype=torch.float32, device="cuda")
    net.forward(xb, y)
    cap = {}
    for k, (name, l) in enumerate(zip(names, layers[:-1])):
        s = P >> _level(name)
        for kind, c in ((0, l["cin"]), (1, l["cout"]), (2, l["cout"])):
            cap[name, kind] = _bf16(net.captured(k, kind, (1, s, s, s, c)))
    net.capture(False)
    # two Adam updates
    steps = []
    w_prev = flat.copy()
    for t in (1, 2):
        net.train_step(xb, target, weight, lr=1e-3)
        gt = np.zeros(net.n_params, np.float32)
        wt = np.zeros(net.n_params, np.float32)
        net.params(get=wt, grads=gt)
        m1, m2, cnt = net.adam_state()
        steps.append(dict(w_prev=w_prev, g=gt, w=wt, m1=m1, m2=m2, t=cnt))
        w_prev = wt
    net.close()
    out = dict(names=names, layers=layers, flat=flat, grads=g0, cap=cap, loss=loss,
               x=xb.float().cpu().numpy().astype(np.float64), y=y.cpu().numpy().astype(np.float64),
               target=target.cpu().numpy().astype(np.float64), weight=weight.cpu().numpy().astype(np.float64),
               adam=steps, dn=dn)
    return out


def _level(name):
    return int(name[1])


def _bf16(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _w(r, name):
    """Weights [cout, 27, cin] and bias of a layer, from the flat parameter vector."""
    l = r["layers"][r["names"].index(name)]
    w = r["flat"][l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])[:, :27 * l["cin"]]
    return (w.reshape(l["cout"], 27, l["cin"]).astype(np.float64),
            r["flat"][l["b_off"]:l["b_off"] + l["cout"]].astype(np.float64))


def _gw(r, name):
    l = r["layers"][r["names"].index(name)]
    g = r["grads"][l["w_off"]:l["w_off"] + l["cout"] * l["kpad"]].reshape(l["cout"], l["kpad"])
    return g[:, :27 * l["cin"]].reshape(l["cout"], 27, l["cin"]).astype(np.float64), \
        r["grads"][l["b_off"]:l["b_off"] + l["cout"]].astype(np.float64), g[:, 27 * l["cin"]:]


def _close(got, ref, tol, what):
    bad = np.abs(got - ref) > tol
    err = np.abs(np.asarray(got, np.float64) - ref)
    record("layer", what=what, elements=int(np.size(ref)), max_err_over_tol=(err / tol).max(),
           max_err_over_max_ref=err.max() / (np.abs(ref).max() + 1e-300))
    assert not bad.any(), (what, int(bad.sum()), float(np.abs(got - ref)[bad].max()), float(tol[bad].min()))


def test_every_convolution_forward(run):
    r, dn = run, run["dn"]
    for name in r["names"]:
        w, b = _w(r, name)
        X, Y = r["cap"][name, 0], r["cap"][name, 1]
        ref = np.maximum(dn.conv3d(X, w, b), 0.0)
        terms = dn.conv3d(np.abs(X), np.abs(w), np.abs(b))
        K = 27 * X.shape[-1]
        _close(Y, ref, U8 * np.abs(ref) + K * 2.0 ** -22 * terms + 1e-30, name)


def test_kernels_between_forward_convolutions(run):
    r, dn = run, run["dn"]
    cap = r["cap"]
    assert np.array_equal(cap["e0a", 0], r["x"])
    for i in range(4):
        assert np.array_equal(cap[f"e{i}b", 0], cap[f"e{i}a", 1])           # same tensor
        if i < 3:
            # 2x2x2 average pooling, FP32 sum rounded once to BF16
            ref = dn.avgpool2(cap[f"e{i}b", 1])
            _close(cap[f"e{i + 1}a", 0], ref, U8 * np.abs(ref) + 1e-6 * dn.avgpool2(np.abs(cap[f"e{i}b", 1])) + 1e-30,
                   f"pool {i}")
    for i in range(2, -1, -1):
        coarse = cap["e3b", 1] if i == 2 else cap[f"d{i + 1}b", 1]
        ref = np.concatenate([dn.upsample2(coarse), cap[f"e{i}b", 1]], axis=4)
        assert np.array_equal(cap[f"d{i}a", 0], ref), i                      # exact copies
        assert np.array_equal(cap[f"d{i}b", 0], cap[f"d{i}a", 1]), i


def test_every_weight_and_bias_gradient(run):
    r, dn = run, run["dn"]
    for name in r["names"]:
        X, G = r["cap"][name, 0], r["cap"][name, 2]
        dw, db = dn.conv3d_wgrad(X, G)
        sw, sb = dn.conv3d_wgrad(np.abs(X), np.abs(G))
        gw, gb, pad = _gw(r, name)
        K = G.shape[1] * G.shape[2] * G.shape[3]          # voxels summed per entry
        _close(gw, dw, K * 2.0 ** -22 * sw + 1e-30, name + " dW")
        _close(gb, db, K * 2.0 ** -22 * sb + 1e-30, name + " db")
        assert np.all(pad == 0.0), name


def test_kernels_between_backward_convolutions(run):
    """Each layer's masked output gradient from the next layer's, through the
    GPU's own tensors: input gradient (flipped-weight convolution), ReLU
    masks, the split of a decoder input's gradient into its coarse part
    (upsampling adjoint) and skip part, the encoder's sum of the skip gradient
    and the pooling adjoint."""
    r, dn = run, run["dn"]
    cap = r["cap"]

    def dgrad(name):
        w, _ = _w(r, name)
        G = cap[name, 2]
        return dn.conv3d_dgrad(G, w), dn.conv3d_dgrad(np.abs(G), np.abs(w)), 27 * G.shape[-1]

    def mask(name):
        return cap[name, 1] > 0

    # head: dL/dtop = 2 w (y - t)/m * head weights, then d0b's ReLU mask
    l = r["layers"][-1]
    hw = r["flat"][l["w_off"]:l["w_off"] + WIDTHS[0]].astype(np.float64)
    gy = 2.0 * r["weight"] * (r["y"] - r["target"]) / r["y"].size
    ref = gy[..., None] * hw * mask("d0b")
    _close(cap["d0b", 2], ref, U8 * np.abs(ref) + 1e-6 * np.abs(gy[..., None] * hw) + 1e-30, "head")
    # inside a level: a's gradient from b's through b's weights and a's mask
    for i in list(range(3)) + [3]:
        for part in ("d", "e") if i < 3 else ("e",):
            a, b = f"{part}{i}a", f"{part}{i}b"
            d, s, K = dgrad(b)
            ref = d * mask(a)
            _close(cap[a, 2], ref, U8 * np.abs(ref) + K * 2.0 ** -21 * s + 1e-30, a)
    # decoder input gradient -> coarse part (upsampling adjoint, coarse mask)
    for i in range(3):
        d, s, K = dgrad(f"d{i}a")
        cu = d.shape[-1] - WIDTHS[i]
        coarse_name = "e3b" if i == 2 else f"d{i + 1}b"
        if coarse_name == "e3b":
            ref = dn.upsample2_adjoint(d[..., :cu]) * mask("e3b")
            tol = 2 * U8 * (dn.upsample2_adjoint(np.abs(d[..., :cu])) + np.abs(ref)) + \
                K * 2.0 ** -19 * dn.upsample2_adjoint(s[..., :cu]) + 1e-30
            _close(cap["e3b", 2], ref, tol, "e3b from d2a")
        else:
            ref = dn.upsample2_adjoint(d[..., :cu]) * mask(coarse_name)
            tol = 2 * U8 * (dn.upsample2_adjoint(np.abs(d[..., :cu])) + np.abs(ref)) + \
                K * 2.0 ** -19 * dn.upsample2_adjoint(s[..., :cu]) + 1e-30
            _close(cap[coarse_name, 2], ref, tol, f"{coarse_name} from d{i}a")
    # encoder output i < 3: skip part of d_i a's input gradient + pooling adjoint
    # of e_{i+1} a's input gradient, then e_i b's mask
    for i in range(3):
        d, s, K = dgrad(f"d{i}a")
        cu = d.shape[-1] - WIDTHS[i]
        skip, skip_s = d[..., cu:], s[..., cu:]
        dc, sc, Kc = dgrad(f"e{i + 1}a")
        pooled = dn.avgpool2_adjoint(dc)
        ref = (skip + pooled) * mask(f"e{i}b")
        tol = 2 * U8 * (np.abs(skip) + np.abs(pooled) + np.abs(ref)) + \
            max(K, Kc) * 2.0 ** -19 * (skip_s + dn.avgpool2_adjoint(sc)) + 1e-30
        _close(cap[f"e{i}b", 2], ref, tol, f"e{i}b")


def test_adam_updates_match_the_oracle(run):
    """Two Adam updates (Kingma and Ba): master weights and both moments,
    element by element, from the GPU's own gradients, against the FP64
    update rule."""
    dn = run["dn"]
    # the hyperparameters as the GPU holds them (FP32 values)
    f32 = lambda v: float(np.float32(v))
    hp = dict(lr=f32(1e-3), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
    m_prev = v_prev = 0.0
    for k, st in enumerate(run["adam"]):
        assert st["t"] == k + 1
        w, m1, m2 = dn.adam_step(st["w_prev"], st["g"], m_prev, v_prev, k + 1, **hp)
        g = st["g"].astype(np.float64)
        # FP32 arithmetic: a few roundings (2^-24 each) of each quantity
        _close(st["m1"], m1, 1e-6 * (np.abs(m1) + 0.1 * np.abs(g)) + 1e-30, f"m1 step {k + 1}")
        _close(st["m2"], m2, 1e-6 * (np.abs(m2) + 1e-3 * g * g) + 1e-30, f"m2 step {k + 1}")
        # weights: FP32 rounding of w, a few roundings of the update, and an
        # absolute floor of lr 2^-23 for elements whose gradients are so small
        # that FP32 moment arithmetic, not the update rule, sets the error
        step = np.abs(w - st["w_prev"])
        _close(st["w"], w, 2e-7 * np.abs(w) + 2e-6 * step + hp["lr"] * 2.0 ** -23, f"w step {k + 1}")
        moved = np.abs(st["w"].astype(np.float64) - st["w_prev"]) > 0
        assert moved.mean() > 0.5, k                      # the update reached the weights
        m_prev, v_prev = st["m1"].astype(np.float64), st["m2"].astype(np.float64)


def test_loss_matches_the_oracle_on_the_gpu_output(run):
    r = run
    ref = np.sum(r["weight"] * (r["y"] - r["target"]) ** 2) / r["y"].size
    assert abs(r["loss"] / ref - 1) < 1e-5, (r["loss"], ref)
