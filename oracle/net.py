"""FP64 CPU reference of the warm-start encoder-decoder (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA network kernels.  The
paper has no network (Sec. 8 names learned priors as future work); this is the
plain FP64 definition of the one the CUDA library trains, so that its forward
pass, loss and every gradient can be checked element by element.

Network (NCHW here, float64):
  input  x = concat(I (3 channels), R_cluster (3 channels), the cold-start
           shading estimate mean_c I / mean_c R_cluster (1 channel), one-hot
           of the cluster label (K channels)), zero-padded to 16 (K <= 9)
  encoder  level l = 1..4 (widths 32, 64, 96, 128): two 3x3 conv + ReLU; a 2x2
           average pool before levels 2..4
  decoder  levels 3, 2, 1: nearest 2x upsampling, concatenation with the
           encoder output of that level, two 3x3 conv + ReLU
  head     1x1 conv to 2K + 1 channels: K reflectance logits w, T_0, T_1..T_K
  output   R_c = sum_k softmax(w)_k b_kc (b the frame's K x 3 palette),
           r = ln R, T = softplus(T_0..T_K) = ln(1 + exp(.)): the layers are
           non-negative (the non-negativity term of Sec. 5.3); a smooth map
           keeps a gradient where a clip at zero would not
Loss: mean squared error of r over B x 3 x H x W values plus mean squared error
of T over B x (K + 1) x H x W values, with optional factors on the r part, the
T_0 part and the T_1..T_K part.

Weights blob (float32 or float64, flat): for every conv layer in order, W with
shape (C_out, C_in, k, k) then bias (C_out,).
"""
from __future__ import annotations

import numpy as np

IN_PAD = 16


def layer_specs(K: int, widths=(32, 64, 96, 128)):
    """[(name, C_in, C_out, k)] in blob order."""
    w1, w2, w3, w4 = widths
    return [
        ("e1a", IN_PAD, w1, 3), ("e1b", w1, w1, 3),
        ("e2a", w1, w2, 3), ("e2b", w2, w2, 3),
        ("e3a", w2, w3, 3), ("e3b", w3, w3, 3),
        ("e4a", w3, w4, 3), ("e4b", w4, w4, 3),
        ("d3a", w4 + w3, w3, 3), ("d3b", w3, w3, 3),
        ("d2a", w3 + w2, w2, 3), ("d2b", w2, w2, 3),
        ("d1a", w2 + w1, w1, 3), ("d1b", w1, w1, 3),
        ("head", w1, 2 * K + 1, 1),
    ]


def n_params(K, widths=(32, 64, 96, 128)):
    return sum(co * ci * k * k + co for _, ci, co, k in layer_specs(K, widths))


def unpack(blob, K, widths=(32, 64, 96, 128)):
    """dict name -> (W (C_out, C_in, k, k), b (C_out,)) as float64 views of the blob."""
    blob = np.asarray(blob, np.float64)
    out, o = {}, 0
    for name, ci, co, k in layer_specs(K, widths):
        n = co * ci * k * k
        out[name] = (blob[o:o + n].reshape(co, ci, k, k), blob[o + n:o + n + co])
        o += n + co
    assert o == blob.size
    return out


def pack(params, K, widths=(32, 64, 96, 128)):
    return np.concatenate([np.concatenate([params[n][0].ravel(), params[n][1].ravel()])
                           for n, *_ in layer_specs(K, widths)])


def he_init(K, seed, widths=(32, 64, 96, 128)):
    """He-normal weights, zero biases (a seeded host draw, float32 blob)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co, k in layer_specs(K, widths):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), size=co * ci * k * k))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------- layers

def conv(x, W, b):
    """Zero-padded 'same' convolution (cross-correlation), k = 1 or 3."""
    B, C, H, Wd = x.shape
    co, ci, k, _ = W.shape
    assert ci == C
    pad = k // 2
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    y = np.zeros((B, co, H, Wd))
    for ky in range(k):
        for kx in range(k):
            y += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + Wd])
    return y + b[None, :, None, None]


def conv_backward(x, W, gy):
    """Gradients of conv(x, W, b) given dL/dy: (dx, dW, db)."""
    B, C, H, Wd = x.shape
    co, ci, k, _ = W.shape
    pad = k // 2
    xp = np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(k):
        for kx in range(k):
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", gy, xp[:, :, ky:ky + H, kx:kx + Wd])
            dxp[:, :, ky:ky + H, kx:kx + Wd] += np.einsum("oc,bohw->bchw", W[:, :, ky, kx], gy)
    dx = dxp[:, :, pad:pad + H, pad:pad + Wd]
    return dx, dW, gy.sum(axis=(0, 2, 3))


def pool2(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_backward(g):
    B, C, H, W = g.shape
    return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


# ---------------------------------------------------------------- network

def make_input(rgb, rcl, labels=None, K=0):
    """(B, 3, H, W) image, clustered reflectance and (B, H, W) labels in 0..K-1
    -> (B, 16, H, W).  The softmax logits of the head index the palette, so the
    label itself (one-hot) is part of the input."""
    B, _, H, W = rgb.shape
    assert 7 + K <= IN_PAD
    x = np.zeros((B, IN_PAD, H, W))
    x[:, 0:3] = rgb
    x[:, 3:6] = rcl
    x[:, 6] = rgb.mean(axis=1) / rcl.mean(axis=1)
    if labels is not None:
        for k in range(K):
            x[:, 7 + k] = labels == k
    return x


def forward(params, x, palette, K):
    """Returns (r (B,3,H,W), T (B,K+1,H,W), cache for backward)."""
    c = {}

    def block(name_a, name_b, inp):
        ya = conv(inp, *params[name_a])
        za = relu(ya)
        yb = conv(za, *params[name_b])
        zb = relu(yb)
        c[name_a] = (inp, ya)
        c[name_b] = (za, yb)
        return zb

    s1 = block("e1a", "e1b", x)
    s2 = block("e2a", "e2b", pool2(s1))
    s3 = block("e3a", "e3b", pool2(s2))
    s4 = block("e4a", "e4b", pool2(s3))
    d3 = block("d3a", "d3b", np.concatenate([up2(s4), s3], axis=1))
    d2 = block("d2a", "d2b", np.concatenate([up2(d3), s2], axis=1))
    d1 = block("d1a", "d1b", np.concatenate([up2(d2), s1], axis=1))
    h = conv(d1, *params["head"])
    c["head"] = (d1, h)
    c["shapes"] = (s1.shape[1], s2.shape[1], s3.shape[1], s4.shape[1])
    w = h[:, :K]
    wmax = w.max(axis=1, keepdims=True)
    e = np.exp(w - wmax)
    s = e / e.sum(axis=1, keepdims=True)                       # (B, K, H, W)
    R = np.einsum("bkhw,bkc->bchw", s, palette)                 # (B, 3, H, W)
    c["head_out"] = (s, R)
    return np.log(R), softplus(h[:, K:]), c


def loss_and_grads(params, x, palette, K, r_tgt, T_tgt, weights=(1.0, 1.0, 1.0)):
    """L and dL/dparams (same dict layout), and dL/dx.  weights: the factors of
    the r part, the T_0 part and the T_1..T_K part of the loss."""
    r, T, c = forward(params, x, palette, K)
    nr, nT = r.size, T.size
    wT = np.full((1, K + 1, 1, 1), float(weights[2]))
    wT[0, 0] = weights[1]
    L = weights[0] * np.sum((r - r_tgt) ** 2) / nr + np.sum(wT * (T - T_tgt) ** 2) / nT
    gr = weights[0] * 2.0 * (r - r_tgt) / nr
    gT = wT * 2.0 * (T - T_tgt) / nT
    s, R = c["head_out"]
    gR = gr / R                                                  # d ln R / dR
    # R_c = sum_j s_j b_jc ; ds_k/dw_l = s_k (delta_kl - s_l)
    gs = np.einsum("bchw,bkc->bkhw", gR, palette)
    gw = s * (gs - np.sum(gs * s, axis=1, keepdims=True))
    gh = np.concatenate([gw, gT * sigmoid(c["head"][1][:, K:])], axis=1)
    grads = {}
    d1, _ = c["head"]
    g, dW, db = conv_backward(d1, params["head"][0], gh)
    grads["head"] = (dW, db)

    def block_back(name_a, name_b, g):
        za, yb = c[name_b]
        g = g * (yb > 0)
        g, dW, db = conv_backward(za, params[name_b][0], g)
        grads[name_b] = (dW, db)
        inp, ya = c[name_a]
        g = g * (ya > 0)
        g, dW, db = conv_backward(inp, params[name_a][0], g)
        grads[name_a] = (dW, db)
        return g

    w1, w2, w3, w4 = c["shapes"]
    g = block_back("d1a", "d1b", g)
    g_up, g_s1 = g[:, :w2], g[:, w2:]
    g = block_back("d2a", "d2b", up2_backward(g_up))
    g_up, g_s2 = g[:, :w3], g[:, w3:]
    g = block_back("d3a", "d3b", up2_backward(g_up))
    g_up, g_s3 = g[:, :w4], g[:, w4:]
    g = block_back("e4a", "e4b", up2_backward(g_up))
    g = block_back("e3a", "e3b", pool2_backward(g) + g_s3)
    g = block_back("e2a", "e2b", pool2_backward(g) + g_s2)
    gx = block_back("e1a", "e1b", pool2_backward(g) + g_s1)
    return L, grads, gx


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1), in place on float64 arrays."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    w -= lr * mh / (np.sqrt(vh) + eps)
