"""The sampled-parity helper (tests/sampling.py) against whole-lattice oracle
runs: the inner block of the oracle run on a periodic box cut from a larger
periodic lattice equals, bitwise, the same sites of the whole lattice's run,
for boxes that wrap around the lattice's faces, in 2D and 3D, over one and
two LB steps, with a drop and a uniform flow so that every term (advection in
both directions, the force, the Laplacians) is non-zero."""
import numpy as np
import pytest

import oracle as O
from paper_0902_3921_gb300 import inputs as I
from sampling import box_oracle, reach

KW = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5)


def _fields(dims, shape, R, vel, op):
    Ls = shape[::-1]  # (Lx, Ly[, Lz])
    phi = I.drop(dims, *Ls, R=R, phi0=O.phi0_of(op), xi=O.xi_of(op))
    n, u = I.rest(dims, *Ls)
    for k, v in enumerate(vel):
        u[k] += v
    return n, phi, u


@pytest.mark.parametrize("steps", [1, 2])
def test_box_inner_block_is_exact_2d(steps):
    shape, m, W = (70, 84), 2, 64  # (Ly, Lx)
    kw = dict(KW, N=0.3, Q=2.5, m=m)
    op = O.Params(dims=2, Lx=shape[1], Ly=shape[0], **kw)
    n, phi, u = _fields(2, shape, 20, (0.02, -0.015), op)
    full = O.State.create(op, n, phi, u)
    full.run(steps)
    fn, fu = full.moments()
    assert reach(m, steps) < W // 2
    for centre in ((35, 42), (2, 80), (60, 3)):  # middle, across the faces
        inner, bn, bphi, bu = box_oracle(kw, n, phi, u, centre, W, steps)
        ix = np.ix_(*inner)
        assert bphi.size > 0
        assert np.array_equal(bphi, full.phi[ix])
        assert np.array_equal(bn, fn[ix])
        assert np.array_equal(bu, np.stack([fu[k][ix] for k in range(2)]))


def test_box_inner_block_is_exact_3d():
    shape, m, W, steps = (36, 40, 44), 2, 32, 1  # (Lz, Ly, Lx)
    kw = dict(KW, N=1 / 6, Q=1 / 3, m=m)
    op = O.Params(dims=3, Lx=shape[2], Ly=shape[1], Lz=shape[0], **kw)
    n, phi, u = _fields(3, shape, 10, (0.02, -0.01, 0.015), op)
    full = O.State.create(op, n, phi, u)
    full.run(steps)
    fn, fu = full.moments()
    for centre in ((18, 20, 22), (1, 38, 10)):
        inner, bn, bphi, bu = box_oracle(kw, n, phi, u, centre, W, steps)
        ix = np.ix_(*inner)
        assert bphi.shape == (W - 2 * reach(m, steps),) * 3
        assert np.array_equal(bphi, full.phi[ix])
        assert np.array_equal(bn, fn[ix])
        assert np.array_equal(bu, np.stack([fu[k][ix] for k in range(3)]))


def test_box_reach_is_needed():
    """The box's false boundary does change the sites near its faces (so
    exactness of the inner block is not trivial), and every changed site
    lies within the reach of a face."""
    shape, m, W, steps = (64, 64), 2, 48, 1
    kw = dict(KW, N=0.3, Q=2.5, m=m)
    op = O.Params(dims=2, Lx=64, Ly=64, **kw)
    n, phi, u = _fields(2, shape, 18, (0.02, -0.015), op)
    full = O.State.create(op, n, phi, u)
    full.run(steps)
    centre = (32, 40)
    ax = [(c - W // 2 + np.arange(W)) % 64 for c in centre]
    ix = np.ix_(*ax)
    p = O.Params(dims=2, Lx=W, Ly=W, **kw)
    st = O.State.create(p, np.ascontiguousarray(n[ix]), np.ascontiguousarray(phi[ix]),
                        np.ascontiguousarray(np.stack([u[k][ix] for k in range(2)])))
    st.run(steps)
    # the whole box differs somewhere near its faces ...
    assert not np.array_equal(st.phi, full.phi[ix])
    # ... and the differing sites all lie within the reach of a face
    r = reach(m, steps)
    bad = np.argwhere(st.phi != full.phi[ix])
    dist = np.minimum(bad, W - 1 - bad).min(axis=1)
    assert dist.max() < r


def test_box_inner_block_is_exact_3d_m8():
    """The configuration the 256^3 sampled GPU test relies on: D3Q19,
    N = 1/6, Q = 1/3, m = 8, one step, a drop with a uniform flow; a 64^3
    box of a 72^3 lattice, across its faces, keeps its 4^3 inner block exact."""
    shape, m, W, steps = (72, 72, 72), 8, 64, 1
    kw = dict(KW, N=1 / 6, Q=1 / 3, m=m)
    op = O.Params(dims=3, Lx=72, Ly=72, Lz=72, **kw)
    n, phi, u = _fields(3, shape, 18, (0.01, -0.005, 0.007), op)
    full = O.State.create(op, n, phi, u)
    full.run(steps)
    fn, fu = full.moments()
    inner, bn, bphi, bu = box_oracle(kw, n, phi, u, (36 + 18, 36, 70), W, steps)
    ix = np.ix_(*inner)
    assert bphi.shape == (4, 4, 4)
    assert np.array_equal(bphi, full.phi[ix])
    assert np.array_equal(bn, fn[ix])
    assert np.array_equal(bu, np.stack([fu[k][ix] for k in range(3)]))


def test_box_inner_block_is_exact_2d_4096_configuration():
    """The configuration the 4096^2 sampled GPU test relies on: D2Q9 with
    the workload's stencil weights, m = 4, three steps, a 160^2 box of a
    176 x 184 lattice across its faces keeps its 52^2 inner block exact."""
    shape, m, W, steps = (176, 184), 4, 160, 3
    kw = dict(KW, N=0.3, Q=2.5, m=m)
    op = O.Params(dims=2, Lx=shape[1], Ly=shape[0], **kw)
    n, phi, u = _fields(2, shape, 40, (0.003, -0.002), op)
    phi = phi + 0.01 * np.sin(np.arange(shape[1]) / 4.0)[None, :]
    full = O.State.create(op, n, phi, u)
    full.run(steps)
    fn, fu = full.moments()
    for centre in ((88, 92), (170, 5)):
        inner, bn, bphi, bu = box_oracle(kw, n, phi, u, centre, W, steps)
        ix = np.ix_(*inner)
        assert bphi.shape == (52, 52)
        assert np.array_equal(bphi, full.phi[ix])
        assert np.array_equal(bn, fn[ix])
        assert np.array_equal(bu, np.stack([fu[k][ix] for k in range(2)]))
