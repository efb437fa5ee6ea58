"""FP64 CPU reference of the learned-correction network (test infrastructure).

Plain numpy forward and backward of the per-element perceptron
x -> (x - mu)/sigma -> W1 -> GELU -> W2 -> GELU -> W3 -> y with the mean
squared error against (t - mu_t)/sigma_t, written out layer by layer; GELU in
its erf form, gelu(z) = z Phi(z).  The parameter layout is the CUDA
library's: W1[H][n_in], b1[H], W2[H][H], b2[H], W3[n_out][H], b3[n_out].
Pinned by central finite differences of its own loss (tests).
"""
import math

import numpy as np

_erf = np.vectorize(math.erf)


def split(params, n_in, H, n_out):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + n_out * H].reshape(n_out, H); o += n_out * H
    b3 = p[o:o + n_out]; o += n_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16(a):
    """Round float values to bfloat16 (round to nearest even), as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, norm, n_in, H, n_out, weight_round=bf16):
    W1, b1, W2, b2, W3, b3 = split(params, n_in, H, n_out)
    W1, W2, W3 = weight_round(W1), weight_round(W2), weight_round(W3)
    mu, sd = norm[0], norm[1]
    xn = (np.asarray(x, np.float64) - mu) / sd
    z1 = xn @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    y = a2 @ W3.T + b3
    return y, (xn, z1, a1, z2, a2, W1, W2, W3)


def loss_and_grad(params, x, t, norm, n_in, H, n_out, weight_round=bf16):
    """MSE over the batch and all outputs, and its gradient with respect to
    every parameter (the rounded weights are used in all products)."""
    y, (xn, z1, a1, z2, a2, W1, W2, W3) = forward(params, x, norm, n_in, H, n_out, weight_round)
    tn = (np.asarray(t, np.float64) - norm[2]) / norm[3]
    n = y.size
    d = y - tn
    loss = float(np.sum(d * d) / n)
    dy = 2.0 * d / n
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ xn
    gb1 = dz1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad
