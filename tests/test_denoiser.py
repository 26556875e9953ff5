"""The learned denoiser's tensor-core kernels against the FP64 oracle (oracle/denoiser.py).

Tolerances follow the arithmetic.  Inputs are rounded to BF16 on both sides, so the only
differences are the FP32 accumulation (at most K * 2^-22 of the sum of |terms| for K
terms, allowing for the tensor cores' internal accumulation) and, for BF16 outputs, one
rounding (2^-8 relative).  Through the whole network the oracle rounds every stored
activation to BF16 where the kernels do, so the outputs differ only where an FP32-vs-FP64
accumulation difference flips a rounding.  Such flips are not rare: a sum of K = 27 cin
terms carries an FP32 error near K 2^-24 of its value (1e-4 for K = 2592), a few percent
of a BF16 half-ulp, so a few percent of the stored activations differ by one ulp (2^-7
relative) in every layer; over ten layers that compounds to a few 1e-3 relative L2 (bar:
1e-2).  The gradients additionally see the kernels' BF16 storage of activation gradients
(about 2^-9 relative per layer), which the oracle keeps exact.
"""
import numpy as np
import pytest

from oracle import denoiser as od

pytestmark = pytest.mark.gpu

FWD_PAIRS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (48, 16)]
# input-gradient convolutions run the forward kernel with cin and cout swapped
DGRAD_PAIRS = [(co, ci) for ci, co in FWD_PAIRS]


@pytest.fixture(scope="module")
def g():
    from paper_1711_03244_gb300 import build
    build.build()
    import paper_1711_03244_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def bf16(a):
    import torch
    return od.bf16_round(torch.as_tensor(np.asarray(a, dtype=np.float64))).numpy()


def random_params(rng, head=True):
    p = np.zeros(od.param_count())
    k = 0
    for ci, co in od.LAYERS:
        p[k:k + 27 * co * ci] = rng.normal(size=27 * co * ci) * np.sqrt(2.0 / (27 * ci))
        k += 27 * co * ci
        p[k:k + co] = rng.normal(size=co) * 0.05
        k += co
    if head:
        p[k:k + 16] = rng.normal(size=16) * 0.3
        p[k + 16] = 0.1
    return p.astype(np.float32)


@pytest.mark.parametrize("cin,cout", sorted(set(FWD_PAIRS + DGRAD_PAIRS)))
def test_conv_forward_matches_oracle(g, cin, cout):
    import torch
    rng = np.random.default_rng(100 + cin + 7 * cout)
    # 3 warp tiles per row, edges in every direction, a ragged last block
    x = bf16(rng.normal(size=(2, 3, 5, 48, cin)))
    w = bf16(rng.normal(size=(27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.normal(size=cout).astype(np.float32)
    got = g.mcx_debug_conv3d(0, x, w, b).astype(np.float64)
    pre = od.conv3d(torch.tensor(x), torch.tensor(w), torch.tensor(b, dtype=torch.float64)).numpy()
    ref = np.maximum(pre, 0)
    s_abs = od.conv3d(torch.tensor(np.abs(x)), torch.tensor(np.abs(w))).numpy() + np.abs(b)
    bound = 2.0 ** -8 * np.abs(ref) + 1.01 * 27 * cin * 2.0 ** -22 * s_abs
    err = np.abs(got - ref)
    print(f"conv {cin}->{cout}: max err {err.max():.2e}, max err/bound {np.max(err / bound):.2f}")
    assert np.all(err <= bound)
    assert np.array_equal(got, bf16(got))                 # outputs are BF16 values


@pytest.mark.parametrize("shape", [(2, 3, 5, 48), (1, 9, 13, 32)])
def test_input_layer_matches_oracle(g, shape):
    """the direct input layer (one input channel, no medium features): FP32 sums of the 27
    taps of the BF16-rounded input, so the same bound as the tensor-core convolutions"""
    import torch
    rng = np.random.default_rng(500 + shape[-1])
    x = bf16(rng.normal(size=shape + (1,)))
    w = bf16(rng.normal(size=(27, 16, 1)) / np.sqrt(27))
    b = rng.normal(size=16).astype(np.float32)
    got = g.mcx_debug_conv3d(0, x, w, b).astype(np.float64)
    xt, wt = torch.tensor(x), torch.tensor(w)
    ref = np.maximum(od.conv3d(xt, wt, torch.tensor(b, dtype=torch.float64)).numpy(), 0)
    s_abs = od.conv3d(xt.abs(), wt.abs()).numpy() + np.abs(b)
    bound = 2.0 ** -8 * np.abs(ref) + 1.01 * 27 * 2.0 ** -22 * s_abs
    err = np.abs(got - ref)
    print(f"input layer on {shape}: max err/bound {np.max(err / bound):.2f}")
    assert np.all(err <= bound)
    assert np.array_equal(got, bf16(got))


@pytest.mark.parametrize("cin,cout", [(16, 16), (48, 16)])
def test_conv_forward_large_ragged_columns(g, cin, cout):
    """a volume large enough for multi-plane work units, with a depth (36) that leaves a
    ragged last column"""
    import torch
    rng = np.random.default_rng(300 + cin)
    x = bf16(rng.normal(size=(2, 36, 64, 64, cin)).astype(np.float32))
    w = bf16(rng.normal(size=(27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.normal(size=cout).astype(np.float32)
    got = g.mcx_debug_conv3d(0, x, w, b).astype(np.float64)
    xt, wt = torch.tensor(x), torch.tensor(w)
    ref = np.maximum(od.conv3d(xt, wt, torch.tensor(b, dtype=torch.float64)).numpy(), 0)
    s_abs = od.conv3d(xt.abs(), wt.abs()).numpy() + np.abs(b)
    bound = 2.0 ** -8 * np.abs(ref) + 1.01 * 27 * cin * 2.0 ** -22 * s_abs
    err = np.abs(got - ref)
    print(f"conv {cin}->{cout} on 2x36x64x64: max err/bound {np.max(err / bound):.2f}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("cin,cout", FWD_PAIRS)
def test_conv_weight_gradient_matches_oracle(g, cin, cout):
    import torch
    rng = np.random.default_rng(200 + cin + 7 * cout)
    x = bf16(rng.normal(size=(2, 3, 5, 48, cin)))
    dy = bf16(rng.normal(size=(2, 3, 5, 48, cout)))
    got = g.mcx_debug_conv3d(1, x, dy=dy).astype(np.float64)
    ref = np.zeros_like(got)
    s_abs = np.zeros_like(got)
    for t, (dz, dyy, dx) in enumerate(od.tap_offsets()):
        xs = od.shift(torch.tensor(x), dz, dyy, dx).numpy()
        ref[t] = np.einsum("nzyxo,nzyxc->oc", dy, xs)
        s_abs[t] = np.einsum("nzyxo,nzyxc->oc", np.abs(dy), np.abs(xs))
    P = x.shape[0] * x.shape[1] * x.shape[2] * x.shape[3]
    bound = P * 2.0 ** -22 * s_abs
    err = np.abs(got - ref)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"dW {cin}x{cout}: rel L2 {rel:.2e}, max err/bound {np.max(err / bound):.2f}")
    assert np.all(err <= bound)
    assert rel < 1e-5


@pytest.mark.parametrize("cin,cout", [(16, 16), (48, 16), (32, 64)])
def test_conv_weight_gradient_large_ragged_columns(g, cin, cout):
    """a volume with multi-plane work units, a depth (19) that leaves a ragged last column,
    lines (40) that end inside a tile, and several CTAs per channel-group pair"""
    import torch
    rng = np.random.default_rng(400 + cin + 7 * cout)
    x = bf16(rng.normal(size=(2, 19, 40, 64, cin)).astype(np.float32))
    dy = bf16(rng.normal(size=(2, 19, 40, 64, cout)).astype(np.float32))
    got = g.mcx_debug_conv3d(1, x, dy=dy).astype(np.float64)
    ref = np.zeros_like(got)
    s_abs = np.zeros_like(got)
    for t, (dz, dyy, dx) in enumerate(od.tap_offsets()):
        xs = od.shift(torch.tensor(x), dz, dyy, dx).numpy()
        ref[t] = np.einsum("nzyxo,nzyxc->oc", dy, xs, optimize=True)
        s_abs[t] = np.einsum("nzyxo,nzyxc->oc", np.abs(dy), np.abs(xs), optimize=True)
    P = x.shape[0] * x.shape[1] * x.shape[2] * x.shape[3]
    bound = P * 2.0 ** -22 * s_abs
    err = np.abs(got - ref)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"dW {cin}x{cout} on 2x19x40x64: rel L2 {rel:.2e}, max err/bound {np.max(err / bound):.2f}")
    assert np.all(err <= bound)
    assert rel < 1e-5


def _net(g, shape, n, params, n_aux=0):
    d = g.Denoiser(shape, max_batch=n, seed=1, n_aux=n_aux)
    d.set_params(params)
    return d


@pytest.mark.parametrize("n_aux", [0, 2])
def test_network_forward_matches_oracle(g, torch_cuda, n_aux):
    torch = torch_cuda
    rng = np.random.default_rng(11)
    shape, n = (8, 8, 64), 2
    p = random_params(rng)
    x = rng.normal(size=(n,) + shape).astype(np.float32)
    aux = rng.normal(size=(n, n_aux) + shape).astype(np.float32) if n_aux else None
    with _net(g, shape, n, p, n_aux) as d:
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        d.forward(xd, yd, aux=None if aux is None else torch.tensor(aux, device="cuda"))
        d.sync()
        y = yd.cpu().numpy().astype(np.float64)
    a64 = None if aux is None else aux.astype(np.float64)
    ref = od.forward(p.astype(np.float64), x.astype(np.float64), bf16=True, aux=a64).numpy()
    exact = od.forward(p.astype(np.float64), x.astype(np.float64), bf16=False, aux=a64).numpy()
    res_g, res_o = y - x, ref - x                 # the network's own contribution
    rel = np.linalg.norm(res_g - res_o) / np.linalg.norm(res_o)
    rel_exact = np.linalg.norm(exact - ref) / np.linalg.norm(res_o)
    print(f"network forward: residual rel L2 {rel:.2e} (BF16 network vs exact FP64 network "
          f"{rel_exact:.2e}), max abs {np.abs(res_g - res_o).max():.2e} of {np.abs(res_o).max():.2e}")
    assert rel < 1e-2
    assert np.abs(res_g - res_o).max() < 5e-2 * np.abs(res_o).max()


def test_network_forward_unaligned_input_takes_the_padded_path(g, torch_cuda):
    """an input that does not start on a 16-byte boundary (a view one float into its
    storage) runs the padded input layer instead of the direct one, which reads 16-byte
    vectors; both match the oracle"""
    torch = torch_cuda
    rng = np.random.default_rng(13)
    shape, n = (8, 8, 64), 2
    p = random_params(rng)
    x = rng.normal(size=(n,) + shape).astype(np.float32)
    ref = od.forward(p.astype(np.float64), x.astype(np.float64), bf16=True).numpy()
    with _net(g, shape, n, p) as d:
        store = torch.empty(x.size + 1, device="cuda")
        xd = store[1:].view((n,) + shape)
        xd.copy_(torch.tensor(x, device="cuda"))
        assert xd.data_ptr() % 16 != 0
        yd = torch.empty_like(xd)
        d.forward(xd, yd)
        d.sync()
        y = yd.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm((y - x) - (ref - x)) / np.linalg.norm(ref - x)
    print(f"network forward, unaligned input: residual rel L2 {rel:.2e}")
    assert rel < 1e-2


def test_network_gradients_match_oracle(g, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(12)
    shape, n = (8, 8, 64), 2
    p = random_params(rng)
    x = rng.normal(size=(n,) + shape).astype(np.float32)
    t = (x + 0.3 * rng.normal(size=x.shape)).astype(np.float32)
    aux = rng.normal(size=(n, 2) + shape).astype(np.float32)
    with _net(g, shape, n, p, n_aux=2) as d:
        loss = d.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 0.0,
                            aux=torch.tensor(aux, device="cuda"))
        gg = d.grads().astype(np.float64)
        assert np.array_equal(d.params(), p)      # lr = 0: no update
    lo, go = od.loss_and_grads(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), bf16=True,
                               aux=aux.astype(np.float64))
    print(f"loss gpu {loss:.6f} oracle {lo:.6f}")
    assert loss == pytest.approx(lo, rel=1e-4)
    k = 0
    names = []
    for name, (ci, co) in zip(od.NAMES, od.LAYERS):
        names += [(name + ".w", k, k + 27 * ci * co), (name + ".b", k + 27 * ci * co, k + 27 * ci * co + co)]
        k += 27 * ci * co + co
    names += [("hw", k, k + 16), ("hb", k + 16, k + 17)]
    for name, a, b in names:
        ga, gb = gg[a:b], go[a:b]
        rel = np.linalg.norm(ga - gb) / max(np.linalg.norm(gb), 1e-30)
        cos = float(ga @ gb / (np.linalg.norm(ga) * np.linalg.norm(gb) + 1e-30))
        print(f"grad {name:6s}: rel L2 {rel:.2e}, cosine {cos:.6f}")
        assert rel < 3e-2 and cos > 0.999, name


def test_adam_step_matches_oracle(g, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(13)
    shape, n = (8, 8, 64), 1
    p = random_params(rng)
    x = rng.normal(size=(n,) + shape).astype(np.float32)
    t = (x + 0.3 * rng.normal(size=x.shape)).astype(np.float32)
    with _net(g, shape, n, p) as d:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        m = v = np.zeros(p.size)
        cur = p.astype(np.float64)
        for step in (1, 2):
            d.train_step(xd, td, 1e-3)
            gr = d.grads().astype(np.float64)
            cur, m, v = od.adam(cur, gr, m, v, step, 1e-3)
            assert np.allclose(d.params(), cur, rtol=1e-5, atol=1e-7), step


def test_apply_is_encode_forward_decode(g, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(14)
    shape, n = (4, 4, 64), 2
    p = random_params(rng)
    phi = (10.0 ** rng.uniform(-9, 0, size=(n,) + shape)).astype(np.float32)
    phi[0, 0, 0, :5] = 0.0
    aux = torch.tensor(rng.normal(size=(n, 2) + shape).astype(np.float32), device="cuda")
    with _net(g, shape, n, p, n_aux=2) as d:
        pd = torch.tensor(phi, device="cuda")
        out = torch.empty_like(pd)
        d.apply(pd, out, aux=aux)
        x, y, back = torch.empty_like(pd), torch.empty_like(pd), torch.empty_like(pd)
        d.encode(pd, x)
        d.forward(x, y, aux=aux)
        d.decode(y, back)
        torch.cuda.synchronize()
        assert torch.equal(out, back)
        xe = x.cpu().numpy()
        assert np.allclose(xe, od.encode(phi), rtol=0, atol=2e-6)
        d.decode(x, back)
        d.sync()
        dec = back.cpu().numpy()
        assert np.allclose(dec, od.decode(xe.astype(np.float64)), rtol=2e-5, atol=1e-12)


def test_training_reduces_the_loss(g, torch_cuda):
    """Denoising smooth fields: the loss falls well below the noise variance."""
    torch = torch_cuda
    rng = np.random.default_rng(15)
    shape, n = (16, 16, 64), 2
    zz, yy, xx = np.meshgrid(np.arange(16), np.arange(16), np.arange(64), indexing="ij")

    def sample():
        out = np.zeros((n,) + shape)
        for i in range(n):
            for _ in range(3):
                c = rng.uniform([0, 0, 0], [16, 16, 64])
                s = rng.uniform(3, 8)
                out[i] += rng.uniform(-1, 1) * np.exp(-((zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2) / (2 * s * s))
        return out.astype(np.float32)

    with g.Denoiser(shape, max_batch=n, seed=3) as d:
        losses = []
        for step in range(300):
            t = sample()
            x = (t + 0.3 * rng.normal(size=t.shape)).astype(np.float32)
            losses.append(d.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 2e-3))
    first, last = np.mean(losses[:10]), np.mean(losses[-20:])
    print(f"training loss {first:.4f} -> {last:.4f}")
    assert first == pytest.approx(0.09, rel=0.15)        # the untrained network returns x
    assert last < 0.5 * first


def test_rejects_bad_shapes(g, torch_cuda):
    torch = torch_cuda
    with pytest.raises(g.McxError):
        g.Denoiser((8, 8, 48))
    with pytest.raises(g.McxError):
        g.Denoiser((6, 8, 64))
    with g.Denoiser((4, 4, 64), max_batch=1) as d:
        x = torch.zeros((2, 4, 4, 64), device="cuda")
        with pytest.raises(g.McxError):
            d.forward(x, torch.empty_like(x))
        with pytest.raises(ValueError):
            d.set_params(np.zeros(3, np.float32))
    with g.Denoiser((4, 4, 64), max_batch=1, n_aux=2) as d:
        x = torch.zeros((1, 4, 4, 64), device="cuda")
        with pytest.raises(ValueError):
            d.forward(x, torch.empty_like(x))              # the features are missing
    with pytest.raises(g.McxError):
        g.Denoiser((4, 4, 64), n_aux=8)


def test_features_match_oracle(g, torch_cuda):
    import workloads
    torch = torch_cuda
    wl = workloads.c5(1, seed=99)[0]
    lab = torch.tensor(wl.labels, device="cuda")
    out = torch.empty((2,) + wl.labels.shape, device="cuda")
    g.Denoiser.features(lab, wl.media, out)
    ref = od.features(wl.labels, np.asarray(wl.media, dtype=np.float32))
    assert np.allclose(out.cpu().numpy(), ref, rtol=0, atol=2e-6)
    # labels past the table count as exterior
    lab2 = torch.tensor(np.array([0, 1, 9], dtype=np.uint8), device="cuda")
    out2 = torch.empty(6, device="cuda")
    g.Denoiser.features(lab2, wl.media[:2], out2)
    assert np.allclose(out2.cpu().numpy().reshape(2, 3)[:, 2], [-2.0, -3.0])


def test_gather_mirrors_and_transposes(g, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(16)
    shape = (4, 64, 64)
    vols = rng.normal(size=(5,) + shape).astype(np.float32)
    with g.Denoiser(shape, max_batch=8) as d:
        src = torch.tensor(vols, device="cuda")
        idx = np.array([0, 4, 2, 2, 1, 3, 0, 4])
        flags = np.arange(8)
        out = torch.empty((8,) + shape, device="cuda")
        d.gather(src, idx, flags, out)
        got = out.cpu().numpy()
    for s in range(8):
        v = vols[idx[s]]                   # mirrors first, then the transpose
        if flags[s] & 1:
            v = v[:, :, ::-1]
        if flags[s] & 2:
            v = v[:, ::-1, :]
        if flags[s] & 4:
            v = v.transpose(0, 2, 1)
        assert np.array_equal(got[s], v), s


def test_bounded_wait_gives_up_and_reports(g):
    """The pipelines' mbarrier wait on a barrier nothing arrives on gives up after its
    poll limit (and the context stays usable); with the arrival first it succeeds."""
    import time
    t0 = time.time()
    assert g.mcx_debug_wait_timeout(False, 16) is True
    assert time.time() - t0 < 30
    assert g.mcx_debug_wait_timeout(True, 16) is False
    # the device still runs work afterwards
    assert g.mcx_debug_wait_timeout(True, 4) is False
