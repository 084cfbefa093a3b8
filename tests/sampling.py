"""Sampled parity at sizes the oracle cannot run whole (test infrastructure).

The oracle runs on a periodic box of side W cut, with periodic wrap, from the
full periodic lattice around a centre site.  One LB step of the hybrid scheme
reaches a bounded distance: the FD update of phi (Eqs. 32-36) reaches 3 sites
per substep (upwind advection and the central divergence of u* 1, the two
Laplacians of Eq. 36 1 each), so phi(t + 1) depends on phi(t) and u*(t)
within 3m; u*(t) depends on phi(t) within 2 (the half-force shift, F of
Eq. 28 with the stencil gradient of mu); the moments at t + 1 add the force
at t + 1 (2 more, which covers the pull stream's 1): 3m + 4 per step.  An
output at distance more than steps x (3m + 6) (a margin of 2) from the box's
faces therefore depends only on inputs inside the box, which the box's false
periodic boundary has not changed: such sites are exact samples of the full
lattice's evolution.  `test_oracle_boxes`
checks this bound against whole-lattice runs."""
import numpy as np

import oracle as O


def reach(m: int, steps: int) -> int:
    """Distance (in sites, along any axis) that `steps` LB steps with m FD
    substeps can carry information, with a margin of 2 per step."""
    return steps * (3 * m + 6)


def box_axes(shape, centre, W):
    """Per array axis, the W lattice indices of the box around `centre`
    (array axis order: (z, y, x) in 3D, (y, x) in 2D), wrapped."""
    return [(c - W // 2 + np.arange(W)) % L for c, L in zip(centre, shape)]


def box_oracle(op_kw: dict, n, phi, u, centre, W: int, steps: int):
    """Run the oracle `steps` LB steps on the W-box around `centre` of the
    full periodic fields n[shape], phi[shape], u[dims, shape].

    Returns (inner, n, phi, u): `inner` the per-axis global indices of the
    exact inner block, and the oracle's n, phi, u* on it."""
    dims = phi.ndim
    m = op_kw["m"]
    r = reach(m, steps)
    lo, hi = r, W - r
    if hi <= lo:
        raise ValueError(f"box side {W} leaves no exact sites for reach {r}")
    ax = box_axes(phi.shape, centre, W)
    ix = np.ix_(*ax)
    nb, pb = np.ascontiguousarray(n[ix]), np.ascontiguousarray(phi[ix])
    ub = np.ascontiguousarray(np.stack([u[k][ix] for k in range(dims)]))
    if dims == 3:
        p = O.Params(dims=3, Lx=W, Ly=W, Lz=W, **op_kw)
    else:
        p = O.Params(dims=2, Lx=W, Ly=W, **op_kw)
    st = O.State.create(p, nb, pb, ub)
    st.run(steps)
    rn, ru = st.moments()
    sl = (slice(lo, hi),) * dims
    inner = [a[lo:hi] for a in ax]
    return inner, rn[sl], st.phi[sl], ru[(slice(None),) + sl]
