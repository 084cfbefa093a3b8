"""Pins of the FP64 surrogate reference (oracle/surrogate.py): convolution
against a direct loop and a known kernel, gradients against central finite
differences, Adam's first step in closed form, and S(k)/L(t) on fields whose
spectrum is known."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_conv_matches_direct_loop_and_identity():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = S.conv3x3_periodic(x, W, b)
    n, h, w, co = 1, 0, 5, 2
    acc = b[co]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            acc += x[n, (h + dy) % 5, (w + dx) % 6, :] @ W[co, dy + 1, dx + 1, :]
    assert y[n, h, w, co] == pytest.approx(acc, abs=1e-12)
    # a kernel with a single 1 at tap (dy, dx) = (1, -1) is the shift x[h + 1, w - 1]
    Wid = np.zeros((3, 3, 3, 3))
    for c in range(3):
        Wid[c, 2, 0, c] = 1.0
    np.testing.assert_allclose(S.conv3x3_periodic(x, Wid, np.zeros(3)),
                               np.roll(x, shift=(-1, 1), axis=(1, 2)), atol=0)


def _net(rng, chans):
    params = []
    for ci, co in zip(chans[:-1], chans[1:]):
        params.append((rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)),
                       0.1 * rng.standard_normal(co)))
    return params


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    params = _net(rng, [4, 6, 6, 4])
    x = rng.standard_normal((2, 6, 5, 4))
    target = rng.standard_normal((2, 6, 5, 4))
    loss, grads = S.loss_and_grads(params, x, target)
    eps = 1e-6
    for li in range(len(params)):
        W, b = params[li]
        for idx in [(0, 0, 0, 0), (1, 2, 1, 3), (W.shape[0] - 1, 1, 2, W.shape[3] - 1)]:
            Wp = W.copy()
            Wp[idx] += eps
            Wm = W.copy()
            Wm[idx] -= eps
            pp = [p if k != li else (Wp, b) for k, p in enumerate(params)]
            pm = [p if k != li else (Wm, b) for k, p in enumerate(params)]
            fd = (S.loss_and_grads(pp, x, target)[0] - S.loss_and_grads(pm, x, target)[0]) / (2 * eps)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
        bp = b.copy()
        bp[1] += eps
        bm = b.copy()
        bm[1] -= eps
        pp = [p if k != li else (W, bp) for k, p in enumerate(params)]
        pm = [p if k != li else (W, bm) for k, p in enumerate(params)]
        fd = (S.loss_and_grads(pp, x, target)[0] - S.loss_and_grads(pm, x, target)[0]) / (2 * eps)
        assert grads[li][1][1] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_first_step_is_a_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3])
    w, m, v = S.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), t=1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_structure_factor_and_domain_size():
    L = 64
    x = np.arange(L)
    # a single cosine mode of wavenumber 2 pi q / L puts all weight in shell q
    for q in (3, 8):
        phi = np.cos(2 * np.pi * q * x / L)[None, :] * np.ones((L, 1))
        k, Sk = S.structure_factor(phi)
        assert np.argmax(Sk) == q - 1
        assert S.domain_size(phi) == pytest.approx(L / q, rel=1e-12)
