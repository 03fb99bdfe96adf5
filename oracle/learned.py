"""Learned Schur-block preconditioner: a plain FP64 reference of the network.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Not in the paper: the
paper's block-diagonal preconditioner P_D (Eq. prec, Sec. 2.2) applies
S_hat^{-1} = L_hat^{-1} D L_hat^{-T} in its third block; the learned variant
keeps that as the input y and adds a correction

    z = |y| (yn + f(yn)),   yn = y / |y|,

f a 1D convolutional network over the grid (length s, periodic), with the
N+1 time levels as channels: conv -> ReLU -> conv -> ReLU -> conv -> ReLU ->
conv, kernel 5, "same" periodic padding.  It is trained to map y = S_hat^{-1} r
to S^{-1} r with the loss |z - t|^2 / |t|^2, t = S^{-1} r.

Layout: activations [C, s] per sample (C channels, s grid points); weights
W[co, ci, k] with tap k reading position (x + k - 2) mod s; bias b[co].
Parity unpinned for the weights themselves (random init); the forward pass is
pinned by a dense-matrix construction of each convolution and the backward
pass by central finite differences (tests/test_oracle_pins.py).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

KW = 5          # kernel width
HALF = KW // 2  # taps reach x-2 .. x+2


def conv1d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Periodic 'same' convolution: out[co, x] = b[co] + sum_ci sum_k
    W[co, ci, k] in[ci, (x + k - 2) mod s]."""
    C_out = W.shape[0]
    s = x.shape[1]
    out = np.repeat(b[:, None], s, axis=1).astype(np.float64)
    for k in range(KW):
        shifted = np.roll(x, -(k - HALF), axis=1)   # shifted[:, x] = in[:, x + k - 2]
        out += W[:, :, k] @ shifted
    return out


def conv1d_backward(x: np.ndarray, W: np.ndarray, gout: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Gradients of sum(gout * conv1d(x, W, b)) w.r.t. x, W and b."""
    gx = np.zeros_like(x, dtype=np.float64)
    gW = np.zeros_like(W, dtype=np.float64)
    for k in range(KW):
        shifted = np.roll(x, -(k - HALF), axis=1)
        gW[:, :, k] = gout @ shifted.T
        # d/dx of W_k @ roll(x, -(k-2)): roll the back-propagated term the other way
        gx += np.roll(W[:, :, k].T @ gout, (k - HALF), axis=1)
    gb = gout.sum(axis=1)
    return gx, gW, gb


def init_params(channels: int, hidden: int, seed: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Four layers channels -> hidden -> hidden -> hidden -> channels; weights
    uniform in +-1/sqrt(fan_in), biases zero; the last layer scaled by 0.1 so
    that the initial network is a small correction."""
    g = np.random.default_rng(seed)
    dims = [channels, hidden, hidden, hidden, channels]
    params = []
    for li in range(4):
        ci, co = dims[li], dims[li + 1]
        a = 1.0 / np.sqrt(ci * KW)
        W = g.uniform(-a, a, size=(co, ci, KW))
        if li == 3:
            W *= 0.1
        params.append((W, np.zeros(co)))
    return params


def forward(params, y: np.ndarray):
    """z = |y| (yn + f(yn)) for one sample y of shape [C, s]; returns z and the
    cache of layer inputs / pre-activations for the backward pass."""
    nrm = np.linalg.norm(y)
    yn = y / nrm if nrm > 0 else y * 0.0
    acts = [yn]
    pres = []
    h = yn
    for li, (W, b) in enumerate(params):
        a = conv1d(h, W, b)
        pres.append(a)
        h = np.maximum(a, 0.0) if li < 3 else a
        acts.append(h)
    z = nrm * (yn + h)
    return z, (nrm, acts, pres)


def loss(params, y: np.ndarray, t: np.ndarray) -> float:
    z, _ = forward(params, y)
    return float(np.sum((z - t) ** 2) / np.sum(t ** 2))


def backward(params, y: np.ndarray, t: np.ndarray):
    """Loss |z - t|^2 / |t|^2 and its gradients w.r.t. every (W, b)."""
    z, (nrm, acts, pres) = forward(params, y)
    tt = np.sum(t ** 2)
    L = float(np.sum((z - t) ** 2) / tt)
    g = 2.0 * (z - t) / tt * nrm           # d loss / d f(yn)
    grads = [None] * 4
    for li in range(3, -1, -1):
        if li < 3:
            g = g * (pres[li] > 0.0)       # ReLU
        W, _ = params[li]
        gx, gW, gb = conv1d_backward(acts[li], W, g)
        grads[li] = (gW, gb)
        g = gx
    return L, grads


def conv_matrix(W: np.ndarray, s: int) -> np.ndarray:
    """Dense matrix of conv1d without bias on the flattened [C_in * s] input,
    built entry by entry from the definition (a pin for conv1d)."""
    C_out, C_in, _ = W.shape
    M = np.zeros((C_out * s, C_in * s))
    for co in range(C_out):
        for ci in range(C_in):
            for x in range(s):
                for k in range(KW):
                    M[co * s + x, ci * s + (x + k - HALF) % s] += W[co, ci, k]
    return M
