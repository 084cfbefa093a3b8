"""The oracle's OpenMP site loops give the same bits for any thread count
(each site's value is computed by the same operations; no reduction crosses
sites): full LB + FD steps in 2D (printed scheme, T term, body force,
stencil_fd) and 3D, one thread against all cores."""
import os

import numpy as np
import pytest

import oracle as O
from paper_0902_3921_gb300 import inputs as I


@pytest.mark.parametrize("kw", [dict(), dict(T=0.28, g=(1e-4, -2e-4, 0.0), force_steps=3),
                                dict(stencil_fd=1, m=21), dict(adv_variant=1, cubic_at_half=1)])
def test_thread_count_does_not_change_the_bits_2d(kw):
    Lx, Ly = 45, 38
    args = dict(Lx=Lx, Ly=Ly, m=4, a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
    args.update(kw)
    p = O.Params(**args)
    phi = I.drop(2, Lx, Ly, R=10, phi0=O.phi0_of(p), xi=O.xi_of(p))
    n, u = I.rest(2, Lx, Ly)
    u = u + 0.002 * np.sin(np.arange(Lx) / 3.0)[None, None, :]
    out = []
    for threads in (1, max(2, os.cpu_count() or 2)):
        assert O.set_threads(threads) == threads
        st = O.State.create(p, n, phi, u)
        st.run(6)
        out.append((st.f.copy(), st.phi.copy()))
    O.set_threads(0)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_thread_count_does_not_change_the_bits_3d():
    L3 = 14
    p = O.Params(dims=3, Lx=L3, Ly=L3 + 2, Lz=L3 - 1, m=8, N=1 / 6, Q=1 / 3)
    phi = I.drop(3, p.Lx, p.Ly, p.Lz, R=4, phi0=O.phi0_of(p), xi=O.xi_of(p))
    n, u = I.rest(3, p.Lx, p.Ly, p.Lz)
    out = []
    for threads in (1, max(2, os.cpu_count() or 2)):
        O.set_threads(threads)
        st = O.State.create(p, n, phi, u)
        st.run(3)
        out.append((st.f.copy(), st.phi.copy()))
    O.set_threads(0)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
