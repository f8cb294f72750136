"""The learned-gradient network's kernels and its unrolled scheme on the GPU.

Convolutions are checked against the FP64 oracle (oracle.conv) on
BF16-representable inputs and BF16-rounded weights, so the only differences
left are FP32 accumulation order (FP32 outputs: 1e-5 relative L2) and the
final rounding of BF16 outputs (half a BF16 ulp, 2^-9 relative, plus the
accumulation error).  The data-fit gradient A^T(Ax - b) is checked against
the oracle's projector pair (2e-5 relative L2: one forward and one
backprojection, 1e-5 each).  A whole learned step and its gradient are
checked against oracle.learned with the forward activations rounded to BF16
as the network defines them and FP64 gradients: the GPU carries every
gradient as a BF16 pair hi + lo (FP32 precision on BF16 tensor cores), so
what is left is FP32 summation order and the activation rounding decisions
it flips (bounds in the test).
Training reduces the loss and beats the untrained scheme on held-out
phantoms; batched and ragged (uneven-size) inference reproduce the
one-volume results bit for bit."""
import numpy as np
import pytest

import oracle
from conftest import max_rel, rel_l2
from oracle import conv as oconv
from oracle import learned as olearned
from paper_2412_10129_gb300 import inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIRS = [(16, 32), (32, 32), (32, 8), (32, 16), (8, 32), (16, 16)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_10129_gb300 import build
    build.build()
    tg.load()


def lm():
    from paper_2412_10129_gb300 import learned
    return learned


def bf16_input(rng, shape, scale=1.0):
    """Random values that BF16 represents exactly, as (torch bf16 CUDA, float64 numpy)."""
    a = oconv.bf16_round((rng.standard_normal(shape) * scale).astype(np.float32))
    return torch.from_numpy(a).to(torch.bfloat16).cuda(), a.astype(np.float64)


def to_oracle_w(w):
    """[27, cout, cin] kernel layout -> oracle W[kz, ky, kx, cin, cout]."""
    w = np.asarray(w, np.float64)
    return w.reshape(3, 3, 3, w.shape[1], w.shape[2]).transpose(0, 1, 2, 4, 3)


def rand_w(rng, cin, cout):
    w = (rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))).astype(np.float32)
    return torch.from_numpy(w).cuda(), to_oracle_w(oconv.bf16_round(w))


def check_bf16_out(y, ref):
    y = y.float().cpu().numpy().astype(np.float64)
    m = np.abs(ref).max()
    assert np.all(np.abs(y - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * m)


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("shape", [(2, 5, 6, 37), (1, 3, 4, 130)])
def test_conv_forward_matches_oracle(cin, cout, shape):
    rng = np.random.default_rng(cin * 100 + cout + shape[3])
    x, xo = bf16_input(rng, shape + (cin,))
    w, wo = rand_w(rng, cin, cout)
    bias = rng.standard_normal(cout).astype(np.float32) * 0.1
    bt = torch.from_numpy(bias).cuda()
    for relu in (False, True):
        ref = oconv.conv3d(xo, wo, bias, relu=relu)
        y = tg.conv3d(x, w, bt, relu=relu, out_f32=True).cpu().numpy()
        assert rel_l2(y, ref) <= 1e-5
        assert max_rel(y, ref) <= 1e-4
        check_bf16_out(tg.conv3d(x, w, bt, relu=relu), ref)
    y = tg.conv3d(x, w, None, out_f32=True).cpu().numpy()
    assert rel_l2(y, oconv.conv3d(xo, wo)) <= 1e-5


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 8), (32, 16), (16, 16)])
def test_tensor_core_and_mma_paths_agree(cin, cout, monkeypatch):
    """The tcgen05 kernels (default) and the mma.sync kernels
    (TG_CONV_IMPL=mma) both match the oracle; their FP32 outputs differ
    only by summation order."""
    rng = np.random.default_rng(cin + 7 * cout)
    x, xo = bf16_input(rng, (2, 6, 5, 300, cin))
    w, wo = rand_w(rng, cin, cout)
    bias = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).cuda()
    ref = oconv.conv3d(xo, wo, bias.cpu().numpy(), relu=True)
    y_tc = tg.conv3d(x, w, bias, relu=True, out_f32=True)
    tg.device_status()
    monkeypatch.setenv("TG_CONV_IMPL", "mma")
    y_mma = tg.conv3d(x, w, bias, relu=True, out_f32=True)
    monkeypatch.delenv("TG_CONV_IMPL")
    for y in (y_tc, y_mma):
        assert rel_l2(y.cpu().numpy(), ref) <= 1e-5
        assert max_rel(y.cpu().numpy(), ref) <= 1e-4
    assert rel_l2(y_tc.cpu().numpy(), y_mma.cpu().numpy()) <= 1e-5
    tg.device_status()


def test_tensor_core_conv_repeats_bit_for_bit():
    """Many items per CTA (each accumulator buffer reused many times) and
    several volumes per launch: repeated launches agree bit for bit and
    with the oracle on every voxel (a missing ordering between the MMAs,
    the row shifts and the epilogue would corrupt whole rows at random)."""
    rng = np.random.default_rng(29)
    dims = [(9, 40, 250), (7, 33, 130), (11, 21, 37)]
    xs = [bf16_input(rng, (1,) + d + (32,)) for d in dims]
    w, wo = rand_w(rng, 32, 32)
    packed = torch.cat([x.reshape(-1, 32) for x, _ in xs]).contiguous()
    first = tg.conv3d_ragged(packed, dims, w, None, relu=False, out_f32=True)
    for _ in range(4):
        assert torch.equal(tg.conv3d_ragged(packed, dims, w, None, relu=False, out_f32=True), first)
    off = 0
    for (x, xo), d in zip(xs, dims):
        n = int(np.prod(d))
        ref = oconv.conv3d(xo, wo).reshape(-1, 32)
        y = first[off:off + n].cpu().numpy()
        assert max_rel(y, ref) <= 1e-4
        assert torch.equal(tg.conv3d(x, w, None, out_f32=True).reshape(-1, 32), first[off:off + n])
        off += n
    tg.device_status()


def test_conv_single_voxel_and_thin_volumes():
    rng = np.random.default_rng(5)
    for shape in [(1, 1, 1, 1), (1, 1, 1, 129), (3, 2, 1, 3), (1, 1, 9, 1)]:
        x, xo = bf16_input(rng, shape + (32,))
        w, wo = rand_w(rng, 32, 32)
        y = tg.conv3d(x, w, None, out_f32=True).cpu().numpy()
        assert rel_l2(y, oconv.conv3d(xo, wo)) <= 1e-5


def test_ragged_conv_matches_per_volume_and_oracle():
    rng = np.random.default_rng(7)
    dims = [(4, 5, 130), (3, 7, 20), (6, 2, 129), (1, 1, 1)]
    xs = [bf16_input(rng, (1,) + d + (32,)) for d in dims]
    w, wo = rand_w(rng, 32, 16)
    bias = torch.from_numpy(rng.standard_normal(16).astype(np.float32)).cuda()
    packed = torch.cat([x.reshape(-1, 32) for x, _ in xs]).contiguous()
    for out_f32 in (False, True):
        y = tg.conv3d_ragged(packed, dims, w, bias, relu=True, out_f32=out_f32)
        off = 0
        for (x, xo), d in zip(xs, dims):
            n = int(np.prod(d))
            one = tg.conv3d(x, w, bias, relu=True, out_f32=out_f32).reshape(-1, 16)
            assert torch.equal(y[off:off + n], one)
            ref = oconv.conv3d(xo, wo, bias.cpu().numpy(), relu=True).reshape(-1, 16)
            if out_f32:
                assert rel_l2(y[off:off + n].cpu().numpy(), ref) <= 1e-5
            else:
                check_bf16_out(y[off:off + n], ref)
            off += n


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 8)])
def test_conv_backward_data_matches_oracle(cin, cout):
    rng = np.random.default_rng(11 + cin + cout)
    gy, gyo = bf16_input(rng, (2, 4, 5, 131, cout))
    w, wo = rand_w(rng, cin, cout)
    gx = tg.conv3d_backward_data(gy, w)
    check_bf16_out(gx, oconv.conv3d_backward_data(gyo, wo))


def test_grad_split_represents_fp32():
    """hi + lo of tg_grad_split equals the (masked) FP32 gradient to 2^-16
    of its magnitude, hi is its BF16 rounding, and the mask follows act > 0;
    tg_lg_pack_split puts s x in channel 0 only."""
    rng = np.random.default_rng(71)
    g = torch.from_numpy((rng.standard_normal((3, 4, 5, 32)) * 10.0 ** rng.uniform(-6, 3, (3, 4, 5, 32)))
                         .astype(np.float32)).cuda()
    act, acto = bf16_input(rng, (3, 4, 5, 32))
    for a in (None, act):
        hi, lo = tg.grad_split(g, a)
        m = np.ones(g.shape) if a is None else (acto > 0)
        gm = g.cpu().numpy().astype(np.float64) * m
        h = hi.float().cpu().numpy().astype(np.float64)
        s_ = h + lo.float().cpu().numpy().astype(np.float64)
        assert np.all(np.abs(s_ - gm) <= 2.0 ** -16 * np.abs(gm))
        np.testing.assert_array_equal(h, oconv.bf16_round(gm.astype(np.float32)))
    x = torch.from_numpy(rng.standard_normal((2, 3, 4)).astype(np.float32)).cuda()
    for C in (8, 16):
        hi, lo = tg.lg_pack_split(x, C, 0.37)
        tot = hi.float().cpu().numpy().astype(np.float64) + lo.float().cpu().numpy()
        ref = np.float32(0.37) * x.cpu().numpy()
        assert np.all(np.abs(tot[..., 0] - ref) <= 2.0 ** -16 * np.abs(ref))
        assert not np.any(tot[..., 1:])
    t = torch.from_numpy(rng.standard_normal((2, 3, 4, 16)).astype(np.float32)).cuda()
    a = torch.full((2, 3, 4), 1.5, device="cuda")
    b = torch.empty_like(a)
    tg.lg_unpack_f32(t, a, b, 2.0, -3.0, accumulate=True)
    torch.testing.assert_close(a, 1.5 + 2.0 * t[..., 0], rtol=0, atol=0)
    torch.testing.assert_close(b, -3.0 * t[..., 1], rtol=0, atol=0)


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 8)])
def test_split_backward_kernels_match_fp64(cin, cout):
    """The backward kernels on a split FP32 gradient reach FP32 accuracy
    against the FP64 oracle applied to the unrounded gradient (1e-5
    relative L2), where a BF16 gradient would be 2^-9 off per element."""
    rng = np.random.default_rng(23 + cin + cout)
    x, xo = bf16_input(rng, (2, 4, 5, 70, cin))
    gyf = rng.standard_normal((2, 4, 5, 70, cout)).astype(np.float32)
    gyo = gyf.astype(np.float64)
    hi, lo = tg.grad_split(torch.from_numpy(gyf).cuda())
    w, wo = rand_w(rng, cin, cout)
    gx = tg.conv3d_backward_data_split(hi, lo, w).cpu().numpy()
    ref = oconv.conv3d_backward_data(gyo, wo)
    assert rel_l2(gx, ref) <= 1e-5 and max_rel(gx, ref) <= 1e-4
    dw = tg.conv3d_backward_weight_split(x, hi, lo).cpu().numpy()
    assert rel_l2(to_oracle_w(dw), oconv.conv3d_backward_weight(xo, gyo)) <= 1e-5
    db = tg.conv3d_backward_bias_split(hi, lo).cpu().numpy()
    assert rel_l2(db, gyo.sum(axis=(0, 1, 2, 3))) <= 1e-5
    # FP32 accumulation into an existing output
    acc = torch.ones((2, 4, 5, 70, cout), device="cuda")
    tg.conv3d(x, w, None, out=acc, accumulate=True)
    assert rel_l2(acc.cpu().numpy(), 1.0 + oconv.conv3d(xo, wo)) <= 1e-5


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 8)])
def test_conv_backward_weight_and_bias_match_oracle(cin, cout):
    rng = np.random.default_rng(13 + cin + cout)
    x, xo = bf16_input(rng, (2, 5, 6, 70, cin))
    gy, gyo = bf16_input(rng, (2, 5, 6, 70, cout))
    dw = tg.conv3d_backward_weight(x, gy).cpu().numpy()
    ref = oconv.conv3d_backward_weight(xo, gyo)            # [3,3,3,cin,cout]
    assert rel_l2(to_oracle_w(dw), ref) <= 1e-5
    db = tg.conv3d_backward_bias(gy).cpu().numpy()
    assert rel_l2(db, gyo.sum(axis=(0, 1, 2, 3))) <= 1e-5


@pytest.mark.parametrize("cin", [16, 32])
def test_conv_backward_weight_many_items_per_cta(cin):
    """The tensor-core weight gradient keeps its sums in tensor memory over
    all of a CTA's items: a volume with several items per CTA (12 x 14 rows
    of 200 voxels = 3 full 64-voxel chunks and a ragged one per row), two
    volumes, against the FP64 oracle; and the same gradient through the
    mma.sync kernel."""
    import os
    rng = np.random.default_rng(41 + cin)
    x, xo = bf16_input(rng, (2, 12, 14, 200, cin))
    gy, gyo = bf16_input(rng, (2, 12, 14, 200, 32))
    ref = oconv.conv3d_backward_weight(xo, gyo)
    dw = tg.conv3d_backward_weight(x, gy).cpu().numpy()
    assert rel_l2(to_oracle_w(dw), ref) <= 1e-5, rel_l2(to_oracle_w(dw), ref)
    os.environ["TG_CONV_IMPL"] = "mma"
    try:
        dm = tg.conv3d_backward_weight(x, gy).cpu().numpy()
    finally:
        del os.environ["TG_CONV_IMPL"]
    assert rel_l2(to_oracle_w(dm), ref) <= 1e-5
    assert rel_l2(dw, dm) <= 1e-5


def test_elementwise_kernels():
    rng = np.random.default_rng(17)
    g, go = bf16_input(rng, (3, 4, 5, 32))
    a, ao = bf16_input(rng, (3, 4, 5, 32))
    out = tg.relu_backward(g, a).float().cpu().numpy()
    np.testing.assert_array_equal(out, np.where(ao > 0, go, 0.0))
    tg.relu_backward(g, a, out=g)                       # in place
    np.testing.assert_array_equal(g.float().cpu().numpy(), out)

    x = torch.from_numpy(rng.random((2, 3, 4, 5)).astype(np.float32)).cuda()
    gr = torch.from_numpy(rng.standard_normal((2, 3, 4, 5)).astype(np.float32)).cuda()
    for C in (8, 16):
        p = tg.lg_pack(x, gr, C, 3.0, -0.5).float().cpu().numpy()
        np.testing.assert_array_equal(p[..., 0], oconv.bf16_round(3.0 * x.cpu().numpy()))
        np.testing.assert_array_equal(p[..., 1], oconv.bf16_round(np.float32(-0.5) * gr.cpu().numpy()))
        assert not np.any(p[..., 2:])
        p0 = tg.lg_pack(x, None, C).float().cpu().numpy()
        assert not np.any(p0[..., 1:])
    t = tg.lg_pack(x, gr, 16, 1.0, 1.0)
    a = torch.full_like(x, 2.0)
    b = torch.empty_like(x)
    tg.lg_unpack(t, a, b, 2.0, 4.0, accumulate=True)
    tf = t.float()
    torch.testing.assert_close(a, 2.0 + 2.0 * tf[..., 0], rtol=0, atol=0)
    torch.testing.assert_close(b, 4.0 * tf[..., 1], rtol=0, atol=0)
    net = torch.from_numpy(rng.standard_normal((2, 3, 4, 5, 8)).astype(np.float32)).cuda()
    xn = tg.lg_update(x, net, 0.25)
    torch.testing.assert_close(xn, x + 0.25 * net[..., 0], rtol=1e-7, atol=0)


def test_data_gradient_matches_oracle():
    g = inputs.random_geometry((40, 36, 28), (1.0, 1.1, 0.9), (64, 48), (1.3, 1.2), 12, seed=3)
    rng = np.random.default_rng(19)
    x = rng.random((2,) + g.vol_shape).astype(np.float32)
    b = rng.random((2,) + g.proj_shape).astype(np.float32)
    xt, bt = torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda()
    gr = tg.gradient(g, xt, bt).cpu().numpy()
    for k in range(2):
        ref = oracle.backproject(g, oracle.forward(g, x[k]) - b[k])
        assert rel_l2(gr[k], ref) <= 2e-5
    nb = tg.gradient(g, xt[0], None).cpu().numpy()
    ref0 = oracle.backproject(g, oracle.forward(g, x[0]))
    assert rel_l2(nb, ref0) <= 2e-5
    acc = torch.full_like(xt[0], 1.5)
    tg.gradient(g, xt[0], None, out=acc, accumulate=True)
    assert rel_l2(acc.cpu().numpy(), ref0 + 1.5) <= 2e-5
    # host buffers take the same path through staging
    assert rel_l2(tg.gradient(g, x[1], b[1]), oracle.backproject(g, oracle.forward(g, x[1]) - b[1])) <= 2e-5


def _small_problem(seed=0, n=24):
    g = inputs.circular_geometry((n, n, n), (4.0,) * 3, (2 * n, 2 * n), (3.2, 3.2), 15, 1000.0, 1536.0)
    L = lm()
    b, x0, gt = L.make_sample(g, seed, I0=1e4)
    return g, b, x0, gt


@pytest.mark.parametrize("signed", [False, True])
def test_learned_step_matches_oracle(signed):
    """One step and its gradient against oracle.learned: forward activations
    rounded to BF16 on both sides (the network's definition), gradients FP64
    in the oracle and BF16 pairs with FP32 sums on the GPU.  With
    non-negative inputs and weights, biases below zero (so that the ReLU
    masks cut) and a non-negative output gradient no sum cancels; with
    weights and gradients of both signs the sums cancel.  What is left is
    FP32 summation order and the BF16 activation roundings it flips (one
    BF16 ulp, 2^-8 of a value, in a few voxels): 1e-2 in both cases."""
    L = lm()
    g, b, x0, gt = _small_problem(seed=3)
    net = L.LearnedGradient(seed=1, gd_init=False, init_scale=1.0).cuda()
    gen = torch.Generator().manual_seed(2)
    with torch.no_grad():
        for li, (w, c) in enumerate(zip(net.weights, net.biases)):
            cin = 2 if li == 0 else w.shape[2]
            if not signed:
                w.copy_(torch.rand(w.shape, generator=gen).cuda() * (2.0 / (27 * cin)))
                c.copy_(-0.3 * torch.rand(c.shape, generator=gen).cuda())
            else:
                c.copy_(0.1 * torch.randn(c.shape, generator=gen).cuda())
        net.weights[0][:, :, 2:] = 0.0
        net.weights[-1][:, 1:, :] = 0.0
    tol = 1e-2
    if not signed:                     # x >= 0 and b = 0 make A^T(Ax - b) >= 0 as well
        x0 = gt + 0.01
        b = torch.zeros_like(b)
    eta = 1.0 / lm().operator_norm_sq(g)
    sx = 1.0 / L.MU_REF
    x = x0.clone().requires_grad_(True)
    xn = net.step(x[None], b[None], g, eta)[0]
    gb = np.random.default_rng(4).standard_normal(g.vol_shape).astype(np.float32)
    gbar = torch.from_numpy(gb if signed else np.abs(gb)).cuda()
    torch.sum(xn * gbar).backward()
    Ws = [to_oracle_w(oconv.bf16_round(w.detach().cpu().numpy())) for w in net.weights]
    Bs = [c.detach().cpu().numpy().astype(np.float64) for c in net.biases]
    xo = x0.cpu().numpy().astype(np.float64)
    bo = b.cpu().numpy().astype(np.float64)
    ref, _ = olearned.step(g, xo, bo, Ws, Bs, sx, sx * eta, 1.0 / sx, round_act=oconv.bf16_round)
    upd = xn.detach().cpu().numpy() - xo
    errs = {"update": rel_l2(upd, ref - xo)}
    gx, dWs, dBs = olearned.step_backward(g, xo, bo, Ws, Bs, sx, sx * eta, 1.0 / sx, gbar.cpu().numpy(),
                                          round_act=oconv.bf16_round)
    errs["x"] = rel_l2(x.grad.cpu().numpy() - gbar.cpu().numpy(), gx - gbar.cpu().numpy())
    for li in range(5):
        dw = to_oracle_w(net.weights[li].grad.cpu().numpy())
        rw = dWs[li]
        if li == 0:
            dw, rw = dw[:, :, :, :2], rw[:, :, :, :2]   # padded input channels carry zeros
        if li == 4:
            dw, rw = dw[..., :1], rw[..., :1]           # padded output channels are unused
        errs[f"w{li}"] = rel_l2(dw, rw)
        db, rb = net.biases[li].grad.cpu().numpy(), dBs[li]
        if li == 4:
            db, rb = db[:1], rb[:1]
        errs[f"b{li}"] = rel_l2(db, rb)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, errs


def test_gd_init_is_gradient_descent():
    """With its initial weights the network is one gradient step of Eq. 4:
    x - eta A^T(Ax - b), up to the BF16 rounding of the gradient channel."""
    L = lm()
    g, b, x0, gt = _small_problem(seed=5)
    net = L.LearnedGradient(seed=0).cuda()
    eta = 1.0 / lm().operator_norm_sq(g)
    with torch.no_grad():
        xn = net.step(x0[None], b[None], g, eta)[0]
        gd = x0 - eta * tg.gradient(g, x0, b)
    assert rel_l2((xn - x0).cpu().numpy(), (gd - x0).cpu().numpy()) <= 2.0 ** -7


def test_batched_and_ragged_inference_match_single():
    L = lm()
    net = L.LearnedGradient(seed=3, init_scale=1.0).cuda()
    with torch.no_grad():
        net.weights[-1].add_(0.02)
        net.weights[-1][:, 1:, :] = 0.0
    probs = []
    for k, n in enumerate((16, 24, 20)):
        g = inputs.circular_geometry((n, n + 2, n - 3), (4.0,) * 3, (2 * n, 2 * n), (3.2, 3.2), 12, 1000.0, 1536.0)
        b, x0, gt = L.make_sample(g, 40 + k)
        probs.append((g, b, x0, 1.0 / lm().operator_norm_sq(g)))
    with torch.no_grad():
        singles = [net(x0, b, g, steps=3, eta=eta) for g, b, x0, eta in probs]
        rag = L.infer_ragged(net, [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs], steps=3,
                             etas=[p[3] for p in probs])
        for s, r in zip(singles, rag):
            assert torch.equal(s, r)
        g, b, x0, eta = probs[0]
        b2 = torch.stack([b, b.flip(0)])
        x02 = torch.stack([x0, x0.flip(0)])
        both = net(x02, b2, g, steps=3, eta=eta)
        assert torch.equal(both[0], singles[0])
        assert torch.equal(both[1], net(x02[1], b2[1], g, steps=3, eta=eta))


def test_training_improves_on_the_untrained_scheme():
    """A short training run (32^3 at 8 mm, 15 angles, 100 batches of 2
    phantoms) lowers the loss and lifts the held-out PSNR well above both
    the untrained scheme (gradient descent from FDK) and the best plain
    CGLS iterate; the oracle's FP64 data residual of the result stays of the
    order of the FDK start's (the network is trained for the image, not for
    the data fit)."""
    L = lm()
    g = inputs.circular_geometry((32,) * 3, (8.0,) * 3, (64, 64), (6.4, 6.4), 15, 1000.0, 1536.0)
    torch.manual_seed(0)
    net = L.LearnedGradient(seed=0).cuda()
    eta = 1.0 / lm().operator_norm_sq(g)
    test = [L.make_sample(g, 5000 + k) for k in range(3)]

    def score():
        with torch.no_grad():
            return np.mean([L.psnr(net(x0, b, g, steps=5, eta=eta), gt) for b, x0, gt in test])

    before = score()
    losses = L.train(net, g, range(1000, 1200), steps=5, batch=2, lr=3e-4)
    after = score()
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
    assert after > before + 3.0
    b, x0, gt = test[0]
    assert L.psnr(net(x0, b, g, steps=5, eta=eta).detach(), gt) > L.cgls_best(g, b, gt, 30)[0] + 1.0
    with torch.no_grad():
        x = net(x0, b, g, steps=5, eta=eta)
    res = np.linalg.norm(oracle.forward(g, x.cpu().numpy()) - b.cpu().numpy().astype(np.float64))
    res0 = np.linalg.norm(oracle.forward(g, x0.cpu().numpy()) - b.cpu().numpy().astype(np.float64))
    assert np.isfinite(res) and res < 2.0 * res0


def test_tensor_core_conv_splits_large_batches():
    """Uniform batches beyond one tensor map's 32 volumes and ragged batches
    beyond one launch's 16 maps run in several launches with the same
    results as one volume at a time."""
    rng = np.random.default_rng(61)
    w, wo = rand_w(rng, 16, 32)
    x, xo = bf16_input(rng, (40, 3, 4, 35, 16))
    y = tg.conv3d(x, w, None, relu=True)
    for k in (0, 31, 32, 39):
        assert torch.equal(y[k:k + 1], tg.conv3d(x[k:k + 1].contiguous(), w, None, relu=True))
    check_bf16_out(y[35:36], oconv.conv3d(xo[35:36], wo, relu=True))
    dims = [(2 + k % 3, 3, 20 + 7 * k) for k in range(20)]
    xs = [bf16_input(rng, (1,) + d + (16,))[0] for d in dims]
    packed = torch.cat([t.reshape(-1, 16) for t in xs]).contiguous()
    yr = tg.conv3d_ragged(packed, dims, w, None, relu=True)
    off = 0
    for t, d in zip(xs, dims):
        n = int(np.prod(d))
        assert torch.equal(yr[off:off + n], tg.conv3d(t, w, None, relu=True).reshape(-1, 32))
        off += n
    tg.device_status()


def test_conv_bounded_wait_gives_up_and_reports_timeout():
    """With the test hook on, each CTA's epilogue waits on a barrier that
    nothing arrives at: the wait runs out after its budget (1e6 clocks), the
    CTA drains its own copies and MMAs and returns, and tg_device_status
    reports TG_ERR_TIMEOUT once.  With the hook off the next launches
    succeed and reproduce the earlier result bit for bit."""
    rng = np.random.default_rng(83)
    x, xo = bf16_input(rng, (2, 5, 7, 100, 32))
    w, wo = rand_w(rng, 32, 32)
    ref = tg.conv3d(x, w, None, out_f32=True)
    tg.device_status()
    tg.test_conv_wait(True, 1_000_000)
    try:
        tg.conv3d(x, w, None, out_f32=True)
        with pytest.raises(tg.TgError) as info:
            tg.device_status()
        assert info.value.code == 5          # TG_ERR_TIMEOUT
    finally:
        tg.test_conv_wait(False, 0)
    tg.device_status()                       # the flag was cleared by the report
    y = tg.conv3d(x, w, None, out_f32=True)
    tg.device_status()
    assert torch.equal(y, ref)
    assert rel_l2(y.cpu().numpy(), oconv.conv3d(xo, wo)) <= 1e-5
