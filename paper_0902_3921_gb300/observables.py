"""Observables of phase separation used to judge the learned surrogate
against the plain scheme (host-side analysis, numpy): the circularly averaged
structure factor S(k) of phi and the domain size L = 2 pi <S> / <k S>."""
from __future__ import annotations

import numpy as np


def structure_factor(phi: np.ndarray):
    """S(k) averaged over rings |k| in [(j - 1/2) dk, (j + 1/2) dk), j = 1..L/2,
    dk = 2 pi / L, of |FFT(phi - <phi>)|^2 / sites.  Returns (k_j, S_j)."""
    L = phi.shape[-1]
    spec = np.abs(np.fft.fft2(phi - np.mean(phi))) ** 2 / phi.size
    q = np.fft.fftfreq(L) * L  # integer wave numbers
    ring = np.rint(np.hypot(q[None, :], q[:, None])).astype(np.int64)
    jmax = L // 2
    sums = np.zeros(jmax + 1)
    counts = np.zeros(jmax + 1)
    sel = ring <= jmax
    np.add.at(sums, ring[sel], spec[sel])
    np.add.at(counts, ring[sel], 1.0)
    j = np.arange(1, jmax + 1)
    return 2.0 * np.pi * j / L, sums[1:] / np.maximum(counts[1:], 1.0)


def domain_size(phi: np.ndarray) -> float:
    k, S = structure_factor(phi)
    return float(2.0 * np.pi * np.sum(S) / np.sum(k * S))
