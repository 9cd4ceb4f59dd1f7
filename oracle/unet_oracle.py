"""Plain FP64 CPU oracle for the learned warm start of the PDHG reconstruction.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The CUDA library never imports,
links or executes it, and it shares no code, tables or helpers with the CUDA path.
Everything is numpy in float64, written for reading, not speed.

The paper starts Algorithms 1 and 2 from zero.  The learned warm start replaces that start
with a prediction of the converged iterates (u, v, r, s) from the data's backprojection.
This module states the network and its training step:

* ``conv3x3`` / ``conv3x3_backward``: 3x3 cross-correlation with zero padding,
  channels-last (NHWC) activations, weights ``[c_out][ky][kx][c_in]``.
* ``avgpool2`` / ``upsample2`` and their adjoints: 2x2 mean pooling and nearest-neighbour
  2x upsampling.
* ``unet_forward`` / ``unet_backward``: the U-Net of Ronneberger, Fischer and Brox (2015),
  with L levels and C0 channels at level 0.
  - Encoder level l: two ReLU convs with C0 * 2^l channels.  Level 0 reads the input; a
    deeper level reads the mean-pooled output of the level above.
  - Decoder level l (L-2 ... 0): two ReLU convs with C0 * 2^l channels.  Their input is the
    concatenation [upsampled output of level l+1, encoder output of level l].
  - Head: one 3x3 conv to the output channels, without ReLU.
* ``mse_loss``: the channel-weighted mean squared error and its gradient.
* ``adam_step``: the Adam update of Kingma and Ba (2015) with bias correction.

Optional bfloat16 emulation (``bf16=True``) rounds values, to nearest even with 8 mantissa
bits, at the same points where the GPU path stores bfloat16:
- the network input;
- the weights;
- every activation written to memory (conv outputs after ReLU, pooled and upsampled maps);
- the loss gradient and every activation gradient.
All arithmetic between those points stays FP64.

Pins (tests/test_oracle_pins.py):
- the convolution against scipy.signal.correlate2d;
- the backward pass against central finite differences of the forward loss;
- pooling and upsampling against hand-written arrays and their adjoint relation;
- Adam's first step against its closed form lr * g / (|g| + eps), and Adam minimising a
  quadratic.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------------------
# bfloat16 rounding (round to nearest, ties to even, on the float32 bit pattern)
# ---------------------------------------------------------------------------------------


def bf16_round(x):
    """Round to the nearest bfloat16 value (ties to even); returns float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(x, bf16):
    return bf16_round(x) if bf16 else x


# ---------------------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------------------


def conv3x3(x, w, b=None, relu=False):
    """y[n, i, j, o] = b[o] + sum_{ky, kx, c} w[o, ky, kx, c] x[n, i + ky - 1, j + kx - 1, c]
    with x = 0 outside the image; then max(y, 0) if relu.  x: (B, H, W, Ci); w: (Co, 3, 3, Ci)."""
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    y = np.zeros((B, H, W, Co))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nijc,oc->nijo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv3x3_backward(x, w, dz):
    """Gradients of conv3x3 (before any ReLU) given dz = dL/dy:
    dx[n, i, j, c] = sum_{ky, kx, o} w[o, ky, kx, c] dz[n, i - ky + 1, j - kx + 1, o],
    dw[o, ky, kx, c] = sum_{n, i, j} dz[n, i, j, o] x[n, i + ky - 1, j + kx - 1, c],
    db[o] = sum_{n, i, j} dz[n, i, j, o]."""
    B, H, W, Ci = x.shape
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nijo,oc->nijc", dz, w[:, ky, kx, :])
            dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dz, xp[:, ky:ky + H, kx:kx + W, :])
    db = dz.sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, db


def avgpool2(x):
    """Mean over disjoint 2x2 blocks: y[n, i, j, c] = 1/4 sum_{a, b in {0,1}} x[n, 2i+a, 2j+b, c]."""
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_adjoint(dy):
    """Transpose of avgpool2: every input pixel receives 1/4 of its block's gradient."""
    return 0.25 * upsample2(dy)


def upsample2(x):
    """Nearest-neighbour 2x upsampling: y[n, i, j, c] = x[n, i // 2, j // 2, c]."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_adjoint(dy):
    """Transpose of upsample2: the sum over each 2x2 block."""
    return 4.0 * avgpool2(dy)


# ---------------------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------------------


def unet_layout(in_ch, out_ch, base, levels):
    """Names and shapes (c_out, c_in) of the convolutions, in parameter order:
    encoder levels 0 .. L-1 (a, b), decoder levels L-2 .. 0 (a, b), head."""
    ch = [base * 2 ** l for l in range(levels)]
    convs = []
    cin = in_ch
    for l in range(levels):
        convs.append((f"enc{l}a", ch[l], cin))
        convs.append((f"enc{l}b", ch[l], ch[l]))
        cin = ch[l]
    for l in range(levels - 2, -1, -1):
        convs.append((f"dec{l}a", ch[l], ch[l + 1] + ch[l]))
        convs.append((f"dec{l}b", ch[l], ch[l]))
    convs.append(("head", out_ch, ch[0]))
    return convs


def params_unflatten(flat, in_ch, out_ch, base, levels):
    """Split a flat parameter vector into {name: (w, b)}; each conv stores its weights
    [c_out][3][3][c_in] and then its bias [c_out]."""
    out, k = {}, 0
    for name, co, ci in unet_layout(in_ch, out_ch, base, levels):
        nw = co * 9 * ci
        w = np.asarray(flat[k:k + nw], dtype=np.float64).reshape(co, 3, 3, ci)
        k += nw
        b = np.asarray(flat[k:k + co], dtype=np.float64)
        k += co
        out[name] = (w, b)
    if k != len(flat):
        raise ValueError("parameter vector has the wrong length")
    return out


def params_flatten(grads, in_ch, out_ch, base, levels):
    parts = []
    for name, _, _ in unet_layout(in_ch, out_ch, base, levels):
        gw, gb = grads[name]
        parts += [np.ravel(gw), np.ravel(gb)]
    return np.concatenate(parts)


def unet_forward(x, params, levels, bf16=False):
    """Forward pass.  Returns (y, cache).  y is the head output, not rounded (the GPU head
    writes float32).  cache holds each conv's input (under the conv's name), the encoder
    outputs ``e{l}``, the decoder outputs ``d{l}`` and the weights used."""
    cache = {"W": {k: (_q(w, bf16), b) for k, (w, b) in params.items()}}
    W = cache["W"]
    h = _q(x, bf16)
    for l in range(levels):
        if l > 0:
            h = _q(avgpool2(h), bf16)
        cache[f"enc{l}a"] = h
        h = _q(conv3x3(h, *W[f"enc{l}a"], relu=True), bf16)
        cache[f"enc{l}b"] = h
        h = _q(conv3x3(h, *W[f"enc{l}b"], relu=True), bf16)
        cache[f"e{l}"] = h
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([upsample2(h), cache[f"e{l}"]], axis=3)
        cache[f"dec{l}a"] = cat
        h = _q(conv3x3(cat, *W[f"dec{l}a"], relu=True), bf16)
        cache[f"dec{l}b"] = h
        h = _q(conv3x3(h, *W[f"dec{l}b"], relu=True), bf16)
        cache[f"d{l}"] = h
    cache["head"] = h
    return conv3x3(h, *W["head"], relu=False), cache


def unet_backward(dy, cache, levels, bf16=False):
    """Backward pass from dy = dL/dy; returns {name: (dw, db)}.  The derivative of a ReLU
    is taken as [output > 0].  A map that feeds two consumers (an encoder output feeds the
    next level's pooling and the decoder's concatenation) sums their gradients once."""
    W = cache["W"]
    grads = {}

    def back(name, dz):
        dx, dw, db = conv3x3_backward(cache[name], W[name][0], dz)
        grads[name] = (dw, db)
        return _q(dx, bf16)

    g = back("head", _q(dy, bf16))                     # d(output of the top level)
    dskip = {}
    for l in range(levels - 1):                        # decoder, top level first
        g = back(f"dec{l}b", g * (cache[f"d{l}"] > 0))
        gcat = back(f"dec{l}a", g * (cache[f"dec{l}b"] > 0))
        cu = gcat.shape[3] - cache[f"e{l}"].shape[3]
        dskip[l] = gcat[..., cu:]
        g = _q(upsample2_adjoint(gcat[..., :cu]), bf16)   # d(output of level l + 1)
    for l in range(levels - 1, -1, -1):                # encoder, bottom level first
        if l < levels - 1:
            g = _q(dskip[l] + avgpool2_adjoint(g), bf16)
        g = back(f"enc{l}b", g * (cache[f"e{l}"] > 0))
        g = back(f"enc{l}a", g * (cache[f"enc{l}b"] > 0))
    return grads


# ---------------------------------------------------------------------------------------
# loss and optimiser
# ---------------------------------------------------------------------------------------


def mse_loss(y, t, ch_weight):
    """L = sum_{n,i,j,c} w_c (y - t)^2 / (B H W C) and dL/dy."""
    B, H, W, C = y.shape
    cnt = B * H * W * C
    d = y - t
    loss = float(np.sum(ch_weight * d * d) / cnt)
    return loss, 2.0 * ch_weight * d / cnt


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    w <- w - lr mhat / (sqrt(vhat) + eps) with mhat = m / (1 - b1^t), vhat = v / (1 - b2^t)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------------------
# the maps between PDHG states and the network's channels
# ---------------------------------------------------------------------------------------
WARM_V_SCALE = 10.0


def warm_features(g, f, in_ch=8):
    """Network input for data f: c0 = T K^T (S f) with T = 1/(K^T 1), S = 1/(K 1) (zero
    where a sum is zero), c1 = K^T 1 / max K^T 1, other channels 0.  Shape (N, N, in_ch)."""
    from . import pat_oracle as po
    n = g.n
    krow = po.forward(g, np.ones((n, n))).ravel()
    kcol = po.adjoint(g, np.ones((g.n_det, g.n_t))).ravel()
    sf = np.where(krow > 0, np.asarray(f, dtype=np.float64).ravel() / np.where(krow > 0, krow, 1.0), 0.0)
    kt = po.adjoint(g, sf.reshape(g.n_det, g.n_t)).ravel()
    x = np.zeros((n * n, in_ch))
    x[:, 0] = np.where(kcol > 0, kt / np.where(kcol > 0, kcol, 1.0), 0.0)
    x[:, 1] = kcol / kcol.max() if kcol.max() > 0 else 0.0
    return x.reshape(n, n, in_ch)


def warm_state(g, pred, reg, alpha, beta, f):
    """PDHG starting state from the 8 prediction channels (N, N, >= 8):
    u = c0, v = (c1, c2) / WARM_V_SCALE, r = proj_alpha(alpha (c3, c4)),
    s = proj_{alpha beta}(alpha beta (c5, c6, c7)), q = K u - f.
    Returns (x, y) in the solver's flat layouts [u, v] and [q, r, s]."""
    from . import pat_oracle as po
    n = g.n
    c = np.asarray(pred, dtype=np.float64).reshape(n * n, -1)
    u = c[:, 0]
    r = po.proj_ball(alpha * c[:, 3:5].T.reshape(2, n, n), alpha).reshape(2, -1)
    q = po.forward(g, u.reshape(n, n)).ravel() - np.asarray(f, dtype=np.float64).ravel()
    xs, ys = [u], [q, r.ravel()]
    if reg == 1:   # TGV
        v = c[:, 1:3].T / WARM_V_SCALE
        s = po.proj_ball(alpha * beta * c[:, 5:8].T.reshape(3, n, n), alpha * beta).reshape(3, -1)
        xs.append(v.ravel())
        ys.append(s.ravel())
    return np.concatenate(xs), np.concatenate(ys)


def warm_target(n, n_data, x, y, reg, alpha, beta, out_ch=8):
    """Training target from a PDHG state (x, y flat): the inverse normalisation of
    ``warm_state`` (without the projections), shape (N, N, out_ch)."""
    NN = n * n
    t = np.zeros((NN, out_ch))
    t[:, 0] = x[:NN]
    t[:, 3] = y[n_data:n_data + NN] / alpha
    t[:, 4] = y[n_data + NN:n_data + 2 * NN] / alpha
    if reg == 1:
        t[:, 1] = x[NN:2 * NN] * WARM_V_SCALE
        t[:, 2] = x[2 * NN:3 * NN] * WARM_V_SCALE
        ab = alpha * beta
        for k in range(3):
            t[:, 5 + k] = y[n_data + (2 + k) * NN:n_data + (3 + k) * NN] / ab
    return t.reshape(n, n, out_ch)
