"""Pins of the FP64 reference network (CPU): convolution against brute force,
every gradient against central finite differences, the softmax palette head
against its limits, Adam against its closed-form first step."""
import numpy as np
import pytest

from oracle import net

TINY = (4, 4, 4, 4)


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5))
    W = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = net.conv(x, W, b)
    for bb in range(2):
        for o in range(2):
            for i in range(4):
                for j in range(5):
                    s = b[o]
                    for c in range(3):
                        for ky in range(3):
                            for kx in range(3):
                                ii, jj = i + ky - 1, j + kx - 1
                                if 0 <= ii < 4 and 0 <= jj < 5:
                                    s += W[o, c, ky, kx] * x[bb, c, ii, jj]
                    assert y[bb, o, i, j] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_pool_and_upsample_are_adjoint_to_their_backward():
    rng = np.random.default_rng(1)
    x, g = rng.normal(size=(1, 2, 4, 6)), rng.normal(size=(1, 2, 2, 3))
    assert np.vdot(net.pool2(x), g) == pytest.approx(np.vdot(x, net.pool2_backward(g)), rel=1e-12)
    y, h = rng.normal(size=(1, 2, 2, 3)), rng.normal(size=(1, 2, 4, 6))
    assert np.vdot(net.up2(y), h) == pytest.approx(np.vdot(y, net.up2_backward(h)), rel=1e-12)


def test_head_limits():
    """A dominant logit gives that base colour; equal logits give the palette mean."""
    K = 3
    palette = np.array([[[0.2, 0.4, 0.6], [0.5, 0.1, 0.3], [0.9, 0.8, 0.7]]])
    params = net.unpack(np.zeros(net.n_params(K, TINY)), K, TINY)
    x = np.zeros((1, 16, 8, 8))
    r, T, _ = net.forward(params, x, palette, K)
    assert np.allclose(np.exp(r[0, :, 0, 0]), palette[0].mean(axis=0), rtol=1e-12)
    W, b = params["head"]
    b[1] = 60.0
    r, T, _ = net.forward(params, x, palette, K)
    assert np.allclose(np.exp(r[0, :, 3, 3]), palette[0, 1], rtol=1e-12)
    assert np.allclose(T, np.log(2.0), rtol=1e-14)                  # softplus(0)
    b[K] = -30.0                                                     # softplus -> exp for large negative
    _, T, _ = net.forward(params, x, palette, K)
    assert np.allclose(T[:, 0], np.exp(-30.0), rtol=1e-12)
    b[K] = 40.0                                                      # and -> identity for large positive
    _, T, _ = net.forward(params, x, palette, K)
    assert np.allclose(T[:, 0], 40.0, rtol=1e-15)


def _problem(seed=0, K=2, H=8, W=8):
    rng = np.random.default_rng(seed)
    blob = net.he_init(K, seed, TINY).astype(np.float64)
    blob += rng.normal(0, 0.05, size=blob.shape)          # non-zero biases too
    params = net.unpack(blob, K, TINY)
    x = net.make_input(rng.uniform(0.1, 0.9, (1, 3, H, W)), rng.uniform(0.1, 0.9, (1, 3, H, W)),
                       rng.integers(0, K, (1, H, W)), K)
    palette = rng.uniform(0.2, 0.8, (1, K, 3))
    r_t = rng.normal(-0.7, 0.2, (1, 3, H, W))
    T_t = rng.normal(0.3, 0.2, (1, K + 1, H, W))
    return blob, params, x, palette, r_t, T_t


def test_gradients_match_finite_differences():
    K = 2
    blob, params, x, palette, r_t, T_t = _problem(K=K)
    wts = (0.7, 1.3, 4.0)
    L, grads, gx = net.loss_and_grads(params, x, palette, K, r_t, T_t, wts)
    gblob = net.pack(grads, K, TINY)
    rng = np.random.default_rng(7)

    def loss_at(b):
        return net.loss_and_grads(net.unpack(b, K, TINY), x, palette, K, r_t, T_t, wts)[0]

    h = 1e-6
    idx = rng.choice(blob.size, size=40, replace=False)
    # include every layer's first weight and bias
    o = 0
    for _, ci, co, k in net.layer_specs(K, TINY):
        idx = np.append(idx, [o, o + co * ci * k * k])
        o += co * ci * k * k + co
    for i in idx:
        e = np.zeros_like(blob)
        e[i] = h
        fd = (loss_at(blob + e) - loss_at(blob - e)) / (2 * h)
        assert gblob[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i
    for (c, yy, xx) in [(0, 0, 0), (4, 3, 5), (2, 7, 7)]:
        e = np.zeros_like(x)
        e[0, c, yy, xx] = h
        fd = (net.loss_and_grads(params, x + e, palette, K, r_t, T_t, wts)[0] -
              net.loss_and_grads(params, x - e, palette, K, r_t, T_t, wts)[0]) / (2 * h)
        assert gx[0, c, yy, xx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_input_layout():
    rgb = np.full((1, 3, 2, 2), 0.5)
    rcl = np.full((1, 3, 2, 2), 0.25)
    lab = np.array([[[0, 2], [1, 2]]])
    x = net.make_input(rgb, rcl, lab, 3)
    assert np.all(x[:, :3] == 0.5) and np.all(x[:, 3:6] == 0.25) and np.all(x[:, 10:] == 0)
    assert np.all(x[:, 6] == 2.0)                                   # mean I / mean R_cluster
    assert np.array_equal(x[0, 7:10].argmax(axis=0), lab[0]) and np.all(x[0, 7:10].sum(axis=0) == 1)


def test_loss_weights_scale_each_part():
    """Weights (a, b, c) give a L_r + b L_T0 + c L_Tk, and the gradients are linear in them."""
    K = 2
    blob, params, x, palette, r_t, T_t = _problem(K=K)
    parts = []
    for w in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        L, g, _ = net.loss_and_grads(params, x, palette, K, r_t, T_t, w)
        parts.append((L, net.pack(g, K, TINY)))
    L, g, _ = net.loss_and_grads(params, x, palette, K, r_t, T_t, (0.5, 2.0, 3.0))
    assert L == pytest.approx(0.5 * parts[0][0] + 2 * parts[1][0] + 3 * parts[2][0], rel=1e-12)
    assert np.allclose(net.pack(g, K, TINY), 0.5 * parts[0][1] + 2 * parts[1][1] + 3 * parts[2][1], rtol=1e-9,
                       atol=1e-15)
    L1, _, _ = net.loss_and_grads(params, x, palette, K, r_t, T_t)
    assert L1 == pytest.approx(sum(p[0] for p in parts), rel=1e-12)


def test_adam_first_step_is_signed_lr():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    net.adam_step(w, g, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(w, [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=1e-12)
