"""The denoiser's tensor-core convolutions against the FP64 oracle on the same
BF16-rounded operands.

Tolerances follow the arithmetic: products of two BF16 numbers are exact in
FP32, the FP32 accumulation over K terms errs by at most about K 2^-24 of the
sum of |terms|, and a BF16 output adds a rounding of 2^-9 relative."""
import numpy as np
import pytest

from tests.parity_record import record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from oracle import denoise
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return torch, nmdose, denoise


def bf16(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def as64(t):
    return t.float().cpu().numpy().astype(np.float64)


def conv_desc(nm, n, d, h, w, c0, c1, coarse, cout):
    return nm.nm_conv3d_desc(n, d, h, w, c0, c1, coarse, cout)


def weights_padded(torch, w3, kpad):
    # w3 [cout, 27, cin] -> [cout, kpad] with k = tap * cin + ci
    cout, _, cin = w3.shape
    wp = np.zeros((cout, kpad), np.float32)
    wp[:, :27 * cin] = w3.reshape(cout, 27 * cin)
    return bf16(torch, wp)


CASES = [
    # n, d, h, w, c0, c1, coarse, cout
    (1, 8, 8, 8, 8, 0, 0, 16),        # first layer (3 channels padded to 8)
    (2, 5, 19, 17, 24, 0, 0, 16),     # ragged shifted-window tiles, 24 channels (a half 16-chunk)
    (1, 9, 33, 35, 48, 0, 0, 32),
    (2, 6, 7, 9, 16, 0, 0, 32),       # ragged voxel count (756, not a multiple of 128)
    (1, 8, 8, 8, 32, 16, 1, 16),      # decoder: upsampled 32 channels + 16 skip
    (1, 4, 4, 4, 64, 0, 0, 128),
    (1, 4, 6, 4, 128, 64, 1, 64),     # deepest decoder input, 192 channels
    (1, 16, 16, 16, 16, 0, 0, 16),
    (1, 6, 10, 12, 32, 0, 0, 64),     # 64 outputs, ragged tiles
    (2, 24, 64, 64, 16, 0, 0, 16),    # more tiles than SMs: persistent CTAs take several
    (1, 32, 64, 48, 48, 0, 0, 32),    # several tiles per CTA and three chunks per tile
    (2, 10, 21, 19, 16, 0, 0, 48),    # 48 outputs (a decoder input's gradient), ragged tiles
    (1, 8, 20, 18, 96, 0, 0, 32),     # 96 inputs: two groups of three chunks, two passes each
    (2, 6, 10, 12, 64, 32, 1, 32),    # decoder at level 1: its input gradient has 96 channels (2 x 48 per launch)
]


@pytest.fixture(params=["default", "unpacked", "gather"])
def conv_path(request, monkeypatch):
    # "default": single-source convolutions with 16, 32, 48 or 64 outputs take the
    # shifted-window kernel, whose 16-output form puts the three x-taps in one
    # MMA (and whose single-chunk weight gradient the three y-taps);
    # "unpacked": those kernels with one tap per MMA; "gather": the
    # im2col-gather kernel for everything.
    for v in ("NM_CONV_GATHER", "NM_CONV_TILE_UNPACKED", "NM_WGRAD_TILE_UNPACKED"):
        monkeypatch.delenv(v, raising=False)
    if request.param == "gather":
        monkeypatch.setenv("NM_CONV_GATHER", "1")
    elif request.param == "unpacked":
        monkeypatch.setenv("NM_CONV_TILE_UNPACKED", "1")
        monkeypatch.setenv("NM_WGRAD_TILE_UNPACKED", "1")
    return request.param


def wgrad_chain(nm, conv_path, n, d, h, w, c0, c1, coarse, cout, kpad):
    """Longest chain of FP32 additions behind one weight-gradient entry."""
    m = n * d * h * w
    tile = conv_path != "gather" and c1 == 0 and not coarse and c0 % 8 == 0 and cout in (16, 32)
    if tile:
        # per CTA: its tiles x 39 K-steps of 16 voxel rows in TMEM; then 8
        # runs of up to 19 CTAs and the 8 runs (the reduction), and the bias
        # gradient's 256-thread blocks of strided voxels
        tiles = n * -(-d // 2) * -(-h // 16) * -(-w // 16)
        grid = min(tiles, 152)
        chain = -(-tiles // grid) * 39 * 16 + -(-grid // 8) + 8
        bias = -(-m // (256 // (cout // 8) * 256)) + 256 // (cout // 8) + 256
        return max(chain, bias)
    # im2col gather: each split sums its voxels in order, then the splits in order
    mtiles = kpad // 128
    splits = -(-(4 * 152) // mtiles)
    if splits * 64 > m:
        splits = -(-m // 64)
    splits = max(splits, 1)
    per = -(-(-(-m // splits)) // 64) * 64
    return per + splits


@pytest.mark.parametrize("case", CASES)
def test_conv_forward_dgrad_wgrad(env, case, conv_path):
    torch, nm, dn = env
    n, d, h, w, c0, c1, coarse, cout = case
    cin = c0 + c1
    rng = np.random.default_rng(hash(case) % 2 ** 32)
    s0 = (n, d // 2, h // 2, w // 2, c0) if coarse else (n, d, h, w, c0)
    x0 = bf16(torch, rng.normal(size=s0))
    x1 = bf16(torch, rng.normal(size=(n, d, h, w, c1))) if c1 else None
    w3 = bf16(torch, rng.normal(0, 1 / np.sqrt(27 * cin), size=(cout, 27, cin)))
    bias = torch.from_numpy(rng.normal(0, 0.1, cout).astype(np.float32))
    kpad = nm.load().nm_conv3d_kpad(cin)
    assert kpad % 128 == 0 and kpad >= 27 * cin
    wg = weights_padded(torch, w3.float().numpy(), kpad).cuda()
    desc = conv_desc(nm, n, d, h, w, c0, c1, coarse, cout)
    x0g = x0.cuda()
    x1g = x1.cuda() if x1 is not None else None
    # reference input: concatenation at full resolution
    X0 = as64(x0)
    if coarse:
        X0 = dn.upsample2(X0)
    X = np.concatenate([X0, as64(x1)], axis=4) if x1 is not None else X0
    W = as64(w3)

    # forward with bias and ReLU
    y = torch.empty((n, d, h, w, cout), dtype=torch.bfloat16, device="cuda")
    nm.nm_conv3d_fwd(desc, x0g, x1g, wg, bias.cuda(), y, True)
    pre = dn.conv3d(X, W, as64(bias))
    ref = np.maximum(pre, 0)
    absum = dn.conv3d(np.abs(X), np.abs(W)) + np.abs(as64(bias))
    got = as64(y.cpu())
    tol = 2.0 ** -8 * np.abs(ref) + 27 * cin * 2.0 ** -23 * absum + 1e-30
    record("conv", case=case, path=conv_path, op="forward", max_err_over_tol=np.max(np.abs(got - ref) / tol))
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)

    # input gradient
    if cin in (16, 32, 48, 64, 96, 128, 192):
        g = bf16(torch, rng.normal(size=(n, d, h, w, cout)))
        dx = torch.empty((n, d, h, w, cin), dtype=torch.bfloat16, device="cuda")
        nm.nm_conv3d_dgrad(desc, g.cuda(), wg, dx)
        G = as64(g)
        ref = dn.conv3d_dgrad(G, W)
        absum = dn.conv3d_dgrad(np.abs(G), np.abs(W))
        tol = 2.0 ** -8 * np.abs(ref) + 27 * cout * 2.0 ** -23 * absum + 1e-30
        got = as64(dx.cpu())
        record("conv", case=case, path=conv_path, op="dgrad", max_err_over_tol=np.max(np.abs(got - ref) / tol))
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)

    # weight and bias gradients.  BF16 x BF16 products are exact in FP32, so
    # the only error is FP32 accumulation: |err| <= L u sum|terms|, L the
    # longest chain of additions any term goes through (a factor 4 for the
    # tensor core's internal order).  Signed data checks the values; data
    # >= 0 (sum|terms| = the value) checks that every contribution is there
    # exactly once, to ~1e-4 relative.
    if cout in (16, 32, 64, 128):
        m = n * d * h * w
        L = wgrad_chain(nm, conv_path, n, d, h, w, c0, c1, coarse, cout, kpad)
        for signed in (True, False):
            if signed:
                g = bf16(torch, rng.normal(size=(n, d, h, w, cout)))
                xa, xb = x0g, x1g
                XX = X
            else:
                g = bf16(torch, rng.random(size=(n, d, h, w, cout)))
                xa = bf16(torch, rng.random(size=s0)).cuda()
                xb = bf16(torch, rng.random(size=(n, d, h, w, c1))).cuda() if c1 else None
                XA = as64(xa.cpu())
                XA = dn.upsample2(XA) if coarse else XA
                XX = np.concatenate([XA, as64(xb.cpu())], axis=4) if c1 else XA
            dw = torch.full((cout, kpad), 7.0, dtype=torch.float32, device="cuda")
            db = torch.zeros(cout, dtype=torch.float32, device="cuda")
            nm.nm_conv3d_wgrad(desc, xa, xb, g.cuda(), dw, db)
            G = as64(g)
            rdw, rdb = dn.conv3d_wgrad(XX, G)
            adw, adb = dn.conv3d_wgrad(np.abs(XX), np.abs(G))
            got = dw.cpu().numpy().astype(np.float64)
            assert np.all(got[:, 27 * cin:] == 0.0)               # padding columns stay exactly zero
            got3 = got[:, :27 * cin].reshape(cout, 27, cin)
            tol = 4 * L * 2.0 ** -24 * adw + 1e-30
            record("conv", case=case, path=conv_path, op="wgrad", signed=signed,
                   max_err_over_tol=np.max(np.abs(got3 - rdw) / tol))
            assert np.all(np.abs(got3 - rdw) <= tol), (signed, np.max(np.abs(got3 - rdw) / tol))
            tolb = 4 * L * 2.0 ** -24 * adb + 1e-30
            assert np.all(np.abs(db.cpu().numpy() - rdb) <= tolb), (signed, np.max(np.abs(db.cpu().numpy() - rdb) / tolb))


def test_conv_is_deterministic(env):
    torch, nm, dn = env
    n, d, h, w, c0, cout = 1, 16, 16, 16, 16, 32
    rng = np.random.default_rng(9)
    x = bf16(torch, rng.normal(size=(n, d, h, w, c0))).cuda()
    g = bf16(torch, rng.normal(size=(n, d, h, w, cout))).cuda()
    desc = conv_desc(nm, n, d, h, w, c0, 0, 0, cout)
    kpad = nm.load().nm_conv3d_kpad(c0)
    outs = []
    for _ in range(2):
        dw = torch.empty((cout, kpad), dtype=torch.float32, device="cuda")
        nm.nm_conv3d_wgrad(desc, x, None, g, dw)
        outs.append(dw.cpu())
    assert torch.equal(outs[0], outs[1])
