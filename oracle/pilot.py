"""Learned pilot: a small convolutional network that stands in for the
stage-1 estimate -- FP64 oracle of its forward pass, loss and gradients.

TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
benchmark's CPU legs, never by the CUDA library or its binding.  It shares
no code with the CUDA path.

The paper's method has no learned part (Sec. 1 prefers a method that needs
no training); this network is an extension that imitates the method's own
stage 1 (Sec. 3: the first estimate Y1 feeds stage 2's matching and Wiener
filter, Sec. 4).  Readings:

  L1  input: two channels per pixel, the noisy image Z and the noise level
      sigma (a constant plane), so one network serves every sigma.
  L2  sixteen 3 x 3 convolutions with zero padding ("same" size): 2 -> 32,
      fourteen 32 -> 32, 32 -> 1, each with a bias; ReLU after the first
      fifteen (a 33 x 33 receptive field, near the 39 x 39 search window the
      network stands in for).
  L3  the network predicts the residual: pilot = Z - f(Z, sigma).
  L4  loss: mean over pixels of (pilot - Y1)^2, Y1 the method's stage-1
      output for the same noisy image.
  L5  weights W[l][tap][ci][co] with tap = 3 (dy + 1) + (dx + 1); a
      convolution is out[y][x][co] = b[co] + sum_{dy,dx,ci}
      in[y + dy][x + dx][ci] W[tap][ci][co] (cross-correlation).

All arithmetic here is FP64; the GPU path stores weights and the inputs of
its 32 -> 32 convolutions in BF16 and accumulates in FP32.
"""
from __future__ import annotations

import numpy as np

# (input channels, output channels, ReLU after) per layer (reading L2)
LAYERS = [(2, 32, True)] + [(32, 32, True)] * 14 + [(32, 1, False)]


def param_count() -> int:
    return sum(9 * ci * co + co for ci, co, _ in LAYERS)


def unpack(theta):
    """Flat parameter vector -> [(W[9][ci][co], b[co])] in layer order
    (per layer: the weights tap-major, then the biases)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for ci, co, _ in LAYERS:
        w = theta[o:o + 9 * ci * co].reshape(9, ci, co)
        o += 9 * ci * co
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    assert o == theta.size
    return out


def conv(x, w, b):
    """Reading L5 on a stack x[B][H][W][ci] with zero padding."""
    B, H, W, _ = x.shape
    xp = np.zeros((B, H + 2, W + 2, x.shape[3]))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    out = np.broadcast_to(b, (B, H, W, w.shape[2])).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            tap = 3 * (dy + 1) + (dx + 1)
            out += xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :] @ w[tap]
    return out


def conv_input_grad(g, w, shape):
    """d(sum g * conv(x)) / dx for the zero-padded correlation."""
    B, H, W, _ = shape
    gx = np.zeros((B, H + 2, W + 2, w.shape[1]))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            tap = 3 * (dy + 1) + (dx + 1)
            gx[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :] += g @ w[tap].T
    return gx[:, 1:H + 1, 1:W + 1, :]


def conv_weight_grad(g, x):
    """d(sum g * conv(x)) / dW[tap][ci][co] and / db[co]."""
    B, H, W, ci = x.shape
    xp = np.zeros((B, H + 2, W + 2, ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    gw = np.zeros((9, ci, g.shape[3]))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            tap = 3 * (dy + 1) + (dx + 1)
            patch = xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :].reshape(-1, ci)
            gw[tap] = patch.T @ g.reshape(-1, g.shape[3])
    return gw, g.sum(axis=(0, 1, 2))


def inputs(Z, sigma):
    """Reading L1: Z[B][H][W] and sigma[B] -> x[B][H][W][2]."""
    Z = np.asarray(Z, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64).reshape(-1, 1, 1) * np.ones_like(Z)
    return np.stack([Z, s], axis=-1)


def forward(theta, Z, sigma, keep=False):
    """pilot[B][H][W] (readings L1-L3); with keep, also the activations."""
    acts = [inputs(Z, sigma)]
    x = acts[0]
    for (w, b), (_, _, relu) in zip(unpack(theta), LAYERS):
        x = conv(x, w, b)
        if relu:
            x = np.maximum(x, 0.0)
        acts.append(x)
    pilot = np.asarray(Z, dtype=np.float64) - x[..., 0]
    return (pilot, acts) if keep else pilot


def loss(theta, Z, sigma, Y1) -> float:
    """Reading L4."""
    return float(np.mean((forward(theta, Z, sigma) - np.asarray(Y1, dtype=np.float64)) ** 2))


def loss_and_grad(theta, Z, sigma, Y1):
    """Loss and its gradient with respect to the flat parameter vector, by the
    chain rule through the layers in reverse order."""
    pilot, acts = forward(theta, Z, sigma, keep=True)
    Y1 = np.asarray(Y1, dtype=np.float64)
    n = pilot.size
    L = float(np.mean((pilot - Y1) ** 2))
    # pilot = Z - out[..., 0]  ->  dL/dout = -2 (pilot - Y1) / n
    g = (-2.0 / n * (pilot - Y1))[..., None]
    params = unpack(theta)
    grads = [None] * len(LAYERS)
    for li in range(len(LAYERS) - 1, -1, -1):
        w, b = params[li]
        if LAYERS[li][2]:
            g = g * (acts[li + 1] > 0)  # ReLU: the output is positive exactly where the pre-activation is
        gw, gb = conv_weight_grad(g, acts[li])
        grads[li] = (gw, gb)
        if li > 0:
            g = conv_input_grad(g, w, acts[li].shape)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return L, flat


def init_params(seed: int = 11) -> np.ndarray:
    """Starting parameters: the input generator's He-normal draw for these
    layer shapes (weights of deviation sqrt(2 / (9 ci)), zero biases)."""
    from paper_2103_10765_gb300 import synth
    return synth.he_normal_params(seed, [(9 * ci, co) for ci, co, _ in LAYERS])
