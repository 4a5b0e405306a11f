"""Warm-start network on the GPU against the FP64 network oracle (oracle/net.py).

Both sides get the same values: weights, image and palette are rounded to
bfloat16 first (the GPU packs weights and inputs to bf16), so the difference
comes from the GPU's bf16 activations only.  Each layer's output is rounded to
bf16 (relative error <= 2^-9); the FP32 accumulation adds ~2^-24 x sqrt(taps x
C_in).  Over the 15 layers of the forward pass and the 15 of the backward
pass, independent roundings grow like sqrt(30) x 2^-9 ~ 1.1% in relative L2
terms.  A weight gradient is a sum over pixels whose terms partly cancel, which
raises the relative error of a small gradient by the cancellation ratio (up to
5% was seen on deep layers).  The bars (forward 2%, gradients 8% relative L2,
cosine >= 0.996) leave a margin over that but catch any indexing, transposition
or sign mistake, each of which gives O(1) error; an element-wise bar (below)
catches one confined to a few elements.
"""
import numpy as np
import pytest

from oracle import net as N

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WIDTHS = (32, 64, 96, 128)
# Element-wise bars (elem_ratio: error / (|ref| + the field's RMS)).  Forward:
# 15 layers of bf16 rounding (2^-9 each) give about sqrt(15) x 2^-9 = 0.0076 at
# an element; 0.02 (about 10 roundings) leaves a margin over the 0.006 seen.
# Weight gradients: a gradient element is a sum over pixels whose terms cancel,
# most on the deep layers with few pixels (0.6 seen on the coarsest encoder
# layer); 1.0 still fails an element off by its own size plus the field's RMS,
# the signature of a wrong tap, row or channel, which the L2 and cosine bars
# could miss when it is confined to a few elements.
ELEM_FWD = 0.02
ELEM_GRAD = 1.0


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def make_case(K, B, H, W, seed):
    rng = np.random.default_rng(seed)
    blob = N.he_init(K, seed, WIDTHS).astype(np.float64)
    blob += rng.normal(0, 0.02, size=blob.shape)
    blob = bf16(blob)
    rgb = bf16(rng.uniform(0.05, 0.95, (B, 3, H, W)))
    labels = rng.integers(0, K, size=(B, H, W)).astype(np.uint8)
    palette = bf16(rng.uniform(0.15, 0.9, (B, K, 3)))
    rcl = np.stack([palette[b][labels[b]].transpose(2, 0, 1) for b in range(B)])
    r_t = rng.normal(-0.8, 0.3, (B, 3, H, W)).astype(np.float32).astype(np.float64)
    T_t = rng.normal(0.3, 0.2, (B, K + 1, H, W)).astype(np.float32).astype(np.float64)
    return blob, rgb, labels, palette, rcl, r_t, T_t


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def cosine(a, b):
    return float(np.vdot(a, b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


def elem_ratio(a, b):
    """Largest element error against the element's own magnitude plus the
    field's RMS (so that near-zero elements are measured against the field's
    scale, not against zero)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float((np.abs(a - b) / (np.abs(b) + np.sqrt(np.mean(b * b)) + 1e-30)).max())


@pytest.mark.parametrize("K,B,H,W", [(3, 2, 16, 24), (6, 1, 24, 40)])
def test_forward_matches_oracle(K, B, H, W):
    """(2, 16, 24): 768 pixels = 6 full 128-pixel tiles; (1, 24, 40): 960 = 7.5 tiles
    (ragged tail), 15 pixels at the coarsest level."""
    from paper_1908_01961_b300 import gid
    blob, rgb, labels, palette, rcl, _, _ = make_case(K, B, H, W, seed=1)
    net = gid.Net(K, WIDTHS)
    assert net.n_params == N.n_params(K, WIDTHS)
    net.set_weights(blob)
    assert np.array_equal(net.weights().astype(np.float64), blob)
    r, T = net.forward(to_dev(rgb), to_dev(labels, torch.uint8), to_dev(palette))
    torch.cuda.synchronize()
    ro, To, _ = N.forward(N.unpack(blob, K, WIDTHS), N.make_input(rgb, rcl, labels, K), palette, K)
    r, T = r.cpu().numpy(), T.cpu().numpy()
    assert rel_l2(T, To) <= 0.02, rel_l2(T, To)
    assert np.abs(T - To).max() <= 0.05 * np.abs(To).max()
    assert rel_l2(r, ro) <= 0.02, rel_l2(r, ro)
    print(f"forward element ratio: r {elem_ratio(r, ro):.4f}, T {elem_ratio(T, To):.4f}")
    assert elem_ratio(r, ro) <= ELEM_FWD and elem_ratio(T, To) <= ELEM_FWD


@pytest.mark.parametrize("K,B,H,W", [(3, 2, 16, 24), (6, 1, 24, 40)])
def test_gradients_match_oracle(K, B, H, W):
    from paper_1908_01961_b300 import gid
    blob, rgb, labels, palette, rcl, r_t, T_t = make_case(K, B, H, W, seed=2)
    net = gid.Net(K, WIDTHS)
    net.set_weights(blob)
    lw = (0.7, 1.3, 4.0)
    net.set_loss_weights(*lw)
    loss = net.backward(to_dev(rgb), to_dev(labels, torch.uint8), to_dev(palette), to_dev(r_t), to_dev(T_t))
    g = net.grads().astype(np.float64)
    params = N.unpack(blob, K, WIDTHS)
    Lo, grads, _ = N.loss_and_grads(params, N.make_input(rgb, rcl, labels, K), palette, K, r_t, T_t, lw)
    assert loss == pytest.approx(Lo, rel=1e-2)
    go = N.unpack(g, K, WIDTHS)
    worst = (0.0, "")
    for name, *_ in N.layer_specs(K, WIDTHS):
        for part, (gpu, ref) in enumerate(zip(go[name], grads[name])):
            what = f"{name} {'W' if part == 0 else 'b'}"
            assert rel_l2(gpu, ref) <= 0.08, (what, rel_l2(gpu, ref))
            assert cosine(gpu.ravel(), ref.ravel()) >= 0.996, (what, cosine(gpu.ravel(), ref.ravel()))
            worst = max(worst, (elem_ratio(gpu, ref), what))
    print(f"gradient element ratio: worst {worst[0]:.4f} ({worst[1]})")
    assert worst[0] <= ELEM_GRAD, worst


def test_adam_step_matches_oracle_update():
    """Two Adam steps on the GPU gradients equal the oracle's Adam applied to the
    same gradients (FP32 vs FP64 arithmetic on identical inputs)."""
    from paper_1908_01961_b300 import gid
    K, B, H, W = 3, 1, 16, 16
    blob, rgb, labels, palette, _, r_t, T_t = make_case(K, B, H, W, seed=3)
    net = gid.Net(K, WIDTHS)
    net.set_weights(blob)
    w = blob.copy()
    m, v = np.zeros_like(w), np.zeros_like(w)
    args = (to_dev(rgb), to_dev(labels, torch.uint8), to_dev(palette), to_dev(r_t), to_dev(T_t))
    for t in (1, 2):
        net.backward(*args)
        g = net.grads().astype(np.float64)
        net.adam_step(1e-3)
        N.adam_step(w, g, m, v, t, lr=1e-3)
        assert np.abs(net.weights() - w).max() <= 1e-6 + 1e-6 * np.abs(w).max()


def test_training_reduces_the_loss():
    from paper_1908_01961_b300 import gid
    K, B, H, W = 4, 2, 32, 32
    blob, rgb, labels, palette, _, _, _ = make_case(K, B, H, W, seed=4)
    rng = np.random.default_rng(5)
    # a learnable target: T a smooth function of the image, r the log palette colour
    T_t = np.repeat(rgb.mean(axis=1, keepdims=True), K + 1, axis=1) * rng.uniform(0.5, 1.5, (1, K + 1, 1, 1))
    r_t = np.log(np.stack([palette[b][labels[b]].transpose(2, 0, 1) for b in range(B)]))
    net = gid.Net(K, WIDTHS, seed=7)
    args = (to_dev(rgb), to_dev(labels, torch.uint8), to_dev(palette), to_dev(r_t), to_dev(T_t))
    first = net.backward(*args)
    net.adam_step(2e-3)
    for _ in range(150):
        net.train_step(*args, lr=2e-3)
    last = net.backward(*args)
    assert last < 0.25 * first, (first, last)


def test_invalid_arguments():
    from paper_1908_01961_b300 import gid
    with pytest.raises(gid.GidError) as e:
        gid.Net(10)                                    # the input holds 7 + K <= 16 channels
    assert e.value.code == -1
    with pytest.raises(gid.GidError):
        gid.Net(3, (32, 48, 96, 128))
    net = gid.Net(3)
    with pytest.raises(gid.GidError):
        net.set_loss_weights(1.0, -1.0, 1.0)
    x = torch.zeros((1, 3, 12, 16), device="cuda")
    with pytest.raises(gid.GidError) as e:
        net.forward(x, torch.zeros((1, 12, 16), dtype=torch.uint8, device="cuda"), torch.ones((1, 3, 3), device="cuda"))
    assert e.value.code == -1


def test_learned_init_is_the_network_output_then_one_base_colour_step():
    """gid_init_learned: state = the network's (r, T) on the frame with palette =
    the initial base colours (bit-equal to gid_net_forward, indirect values below
    zero_below set to 0), T_0 refit to the data term (oracle: fit_direct), then b = b_init +
    Delta b from the base-colour step on those layers (oracle: SVD solve)."""
    import oracle as O
    from harness import Case
    from paper_1908_01961_b300 import gid
    case = Case(H=48, W=64, K=4, n_cells=12, seed=0)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    net = gid.Net(case.K, seed=3)
    zb = 0.004
    s.init_learned(net, zb)
    X = s.state()
    pal = torch.from_numpy(case.b_init.astype(np.float32)).cuda()[None].contiguous()
    r, T = net.forward(rgb[None].contiguous(), lab[None].contiguous(), pal)
    torch.cuda.synchronize()
    X = X.cpu().numpy()
    T = T[0].cpu().numpy()
    T[1:][T[1:] < zb] = 0.0                               # indirect values below zero_below start at zero
    assert np.array_equal(X[:3], r[0].cpu().numpy()) and np.array_equal(X[4:], T[1:])
    Xn = np.concatenate([r[0].cpu().numpy(), T]).astype(np.float64)
    T0 = O.fit_direct(case.frames[0].I.astype(np.float32), Xn, case.b_init)[3]
    assert np.abs(X[3] - T0).max() <= 1e-5 * max(1.0, np.abs(T0).max())
    pb = case.oracle_problem()
    A, g = pb.dense_normal(X.astype(np.float64))
    b_ref = case.b_init + O.dense_solve(A, g)
    assert np.abs(s.base_colors() - b_ref).max() <= 1e-3
    with pytest.raises(gid.GidError):
        s.init_learned(gid.Net(3))                       # K mismatch
    with pytest.raises(gid.GidError):
        s.init_learned(net, -1.0)
