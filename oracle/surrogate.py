"""FP64 reference of the learned surrogate: a stack of periodic 3x3
convolutions (ReLU between layers, none after the last), its gradients, the
MSE loss, one Adam step, and the observables that compare the surrogate with
the plain scheme (structure factor S(k), domain size L(t), mass drift).

TEST INFRASTRUCTURE ONLY (the tests, the package smoke check and the CPU
baseline legs of bench.py): plain numpy, written from the definitions, no
blocking or fusion; shares no code with the CUDA library.

Layouts: activations NHWC [N][H][W][C]; a layer's weights [Cout][3][3][Cin]
(tap index (dy + 1, dx + 1)), biases [Cout].  The convolution is periodic:
    y[n, h, w, co] = b[co] + sum_{dy, dx, ci} x[n, h + dy, w + dx, ci] W[co, dy+1, dx+1, ci]
with indices wrapped.  The paper has no counterpart of this network; it is
the learned-surrogate extension, measured with the paper's observables.
"""
from __future__ import annotations

import numpy as np


def conv3x3_periodic(x, W, b):
    """Forward convolution, FP64."""
    N, H, Wd, Ci = x.shape
    Co = W.shape[0]
    y = np.broadcast_to(b.astype(np.float64), (N, H, Wd, Co)).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))  # xs[h, w] = x[h + dy, w + dx]
            y += np.einsum("nhwc,oc->nhwo", xs, W[:, dy + 1, dx + 1, :])
    return y


def conv3x3_periodic_backward(x, W, dy_):
    """Gradients of sum(dy_ * conv(x, W, b)) with respect to x, W and b."""
    N, H, Wd, Ci = x.shape
    dx_ = np.zeros_like(x, dtype=np.float64)
    dW = np.zeros_like(W, dtype=np.float64)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
            dW[:, dy + 1, dx + 1, :] = np.einsum("nhwo,nhwc->oc", dy_, xs)
            contrib = np.einsum("nhwo,oc->nhwc", dy_, W[:, dy + 1, dx + 1, :])
            dx_ += np.roll(contrib, shift=(dy, dx), axis=(1, 2))
    db = dy_.sum(axis=(0, 1, 2))
    return dx_, dW, db


def forward(params, x):
    """params: list of (W, b).  Returns the output and the per-layer inputs and
    pre-activations needed by backward()."""
    acts, pres = [], []
    a = x
    for li, (W, b) in enumerate(params):
        acts.append(a)
        z = conv3x3_periodic(a, W, b)
        pres.append(z)
        a = np.maximum(z, 0.0) if li < len(params) - 1 else z
    return a, acts, pres


def mse(y, target):
    return float(np.mean((y - target) ** 2))


def loss_and_grads(params, x, target):
    """MSE loss of the network output against target and its gradients."""
    y, acts, pres = forward(params, x)
    loss = mse(y, target)
    dz = 2.0 * (y - target) / y.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        dx, dW, db = conv3x3_periodic_backward(acts[li], W, dz)
        grads[li] = (dW, db)
        if li > 0:
            dz = dx * (pres[li - 1] > 0)
    return loss, grads


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) at step t >= 1; returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def structure_factor(phi):
    """Shell-averaged S(k) = <|FFT(phi - mean)|^2> / sites over |k| shells of
    width 2 pi / L (square periodic lattice).  Returns (k, S)."""
    L = phi.shape[0]
    f = np.fft.fft2(phi - phi.mean())
    p = (np.abs(f) ** 2) / phi.size
    k1 = 2.0 * np.pi * np.fft.fftfreq(L)
    kx, ky = np.meshgrid(k1, k1, indexing="xy")
    kmag = np.sqrt(kx * kx + ky * ky)
    shell = np.rint(kmag / (2.0 * np.pi / L)).astype(int)
    nb = L // 2
    S = np.bincount(shell.ravel(), weights=p.ravel(), minlength=nb + 1)[1:nb + 1]
    cnt = np.bincount(shell.ravel(), minlength=nb + 1)[1:nb + 1]
    k = 2.0 * np.pi * np.arange(1, nb + 1) / L
    return k, S / np.maximum(cnt, 1)


def domain_size(phi):
    """L(t) = 2 pi sum_k S(k) / sum_k k S(k)."""
    k, S = structure_factor(phi)
    return float(2.0 * np.pi * S.sum() / (k * S).sum())
