"""Pins of the oracle's operators against what the paper and mathematics fix.

Covers stencils (Eqs. 30-31, their Taylor expansions Eqs. 37-39 and exact
Fourier symbols), the equilibrium and forcing moments (Eqs. 13-16, 20, 26),
the FD operators (Eqs. 32-36) through exact amplification factors, and the
dense-matrix brute force on tiny periodic grids.
"""
import numpy as np
import pytest

import oracle as O


def _params(dims, Lx, Ly, Lz=1, **kw):
    return O.Params(dims=dims, Lx=Lx, Ly=Ly, Lz=Lz if dims == 3 else 1, **kw)


def _coords(p):
    shp = p.shape
    g = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shp], indexing="ij")
    return g[::-1]  # x, y(, z)


def _interior(p, margin=2):
    c = _coords(p)
    L = [p.Lx, p.Ly, p.Lz][: p.dims]
    m = np.ones(p.shape, dtype=bool)
    for a in range(p.dims):
        m &= (c[a] >= margin) & (c[a] <= L[a] - 1 - margin)
    return m


# ---- c1: stencils exact on polynomials (Eqs. 30-31, Taylor form Eqs. 37-38) ----

@pytest.mark.parametrize("N,Q", [(0.5, 1.0), (0.3, 2.5), (1 / 3, 2 / 3), (7 / 12, 7 / 6)])
def test_stencil_2d_polynomials(N, Q):
    p = _params(2, 16, 16, N=N, Q=Q)
    x, y = _coords(p)
    m = _interior(p)
    # first derivative: exact on x, x^3 picks up (1/6) dx^3 -> +1, x y^2 picks up
    # (1-2N)/2 dx dy^2 -> 1 - 2N  (Eq. 37)
    gx = O.grad_D(p, x)[0]
    np.testing.assert_allclose(gx[m], 1.0, rtol=0, atol=1e-12)
    gy = O.grad_D(p, y)[1]
    np.testing.assert_allclose(gy[m], 1.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.grad_D(p, x ** 3)[0][m], (3 * x ** 2 + 1)[m], atol=1e-10)
    np.testing.assert_allclose(O.grad_D(p, x * y ** 2)[0][m], (y ** 2 + 1 - 2 * N)[m], atol=1e-10)
    np.testing.assert_allclose(O.grad_D(p, y * x ** 2)[1][m], (x ** 2 + 1 - 2 * N)[m], atol=1e-10)
    # the transposed stencil gives no cross talk: d_Dy of a function of x is 0
    np.testing.assert_allclose(O.grad_D(p, x ** 3)[1][m], 0.0, atol=1e-10)
    # Laplacian: exact on x^2 + y^2; x^4 picks up (1/12) dx^4 -> +2; x^2 y^2 picks up
    # the mixed term of Eq. 38, read as (1-Q)/2 dx^2 dy^2 (the printed dy^3 is a typo)
    np.testing.assert_allclose(O.lap_D(p, x ** 2 + y ** 2)[m], 4.0, atol=1e-11)
    np.testing.assert_allclose(O.lap_D(p, x ** 4)[m], (12 * x ** 2 + 2)[m], atol=1e-9)
    np.testing.assert_allclose(O.lap_D(p, x ** 2 * y ** 2)[m],
                               (2 * x ** 2 + 2 * y ** 2 + 2 * (1 - Q))[m], atol=1e-9)
    # uniform field: every operator gives exactly 0
    one = np.full(p.shape, 0.7)
    assert np.all(O.grad_D(p, one) == 0.0 * one) or np.max(np.abs(O.grad_D(p, one))) < 1e-15
    assert np.max(np.abs(O.lap_D(p, one))) < 1e-15


def test_stencil_taylor_coefficients_eq39():
    """d_Dx(lap_D) applied to x^3 y^2 and x y^4 reproduces the bracketed
    coefficients of Eq. 39 (with the corrected mixed term of Eq. 38)."""
    for N, Q in [(0.5, 1.0), (0.3, 2.5), (7 / 12, 7 / 6)]:
        p = _params(2, 24, 24, N=N, Q=Q)
        x, y = _coords(p)
        m = _interior(p, margin=3)
        for f, d_exact, c5, c32, c14 in [
            # f, d_x lap f, and the coefficient of dx^5, dx^3 dy^2, dx dy^4 applied to f
            (x ** 3 * y ** 2, 6 * y ** 2 + 6 * x ** 2 + 0 * x, 0.0, 12.0, 0.0),
            (x * y ** 4, 12 * y ** 2, 0.0, 0.0, 24.0),
            (x ** 5, 60 * x ** 2, 120.0, 0.0, 0.0),
        ]:
            got = O.grad_D(p, O.lap_D(p, f))[0]
            want = (d_exact + 0.25 * c5 + (1 / 6 + (1 - 2 * N) / 2 + (1 - Q) / 2) * c32
                    + (1 / 12 + (1 - 2 * N) / 2) * c14)
            # higher-order terms vanish on these polynomials except for the
            # d_x^3 d_y^2 piece of x^3 y^2 (degree 5); the remaining d_x lap of
            # lower derivative terms are exact.
            np.testing.assert_allclose(got[m], np.broadcast_to(want, p.shape)[m], atol=1e-8)


def test_stencil_3d_polynomials():
    for N, Q in [(0.5, 1.0), (1 / 6, 1 / 3), (0.3, 0.6)]:
        p = _params(3, 10, 11, 12, N=N, Q=Q)
        x, y, z = _coords(p)
        m = _interior(p)
        g = O.grad_D(p, x + 2 * y - 3 * z)
        np.testing.assert_allclose(g[0][m], 1.0, atol=1e-12)
        np.testing.assert_allclose(g[1][m], 2.0, atol=1e-12)
        np.testing.assert_allclose(g[2][m], -3.0, atol=1e-12)
        np.testing.assert_allclose(O.lap_D(p, x ** 2 + y ** 2 + z ** 2)[m], 6.0, atol=1e-10)
        np.testing.assert_allclose(O.lap_D(p, x * y + y * z)[m], 0.0, atol=1e-10)
        np.testing.assert_allclose(O.grad_D(p, x ** 3)[0][m], (3 * x ** 2 + 1)[m], atol=1e-9)


def _fourier_symbols(dims, N, Q, k):
    """Exact symbols of the stencils on exp(i k.r):
    d_Dx -> i sx,  lap_D -> lam."""
    c = np.cos(k)
    s = np.sin(k)
    if dims == 2:
        M = (1 - 2 * N) / 4
        R = (1 - Q) / 2
        sx = 2 * s[0] * (N + 2 * M * c[1])
        sy = 2 * s[1] * (N + 2 * M * c[0])
        lam = 2 * Q * (c[0] + c[1]) + 4 * R * c[0] * c[1] - 4 * (Q + R)
        return (sx, sy), lam
    M = (1 - 2 * N) / 8
    R = (1 - Q) / 4
    sx = 2 * s[0] * (N + 2 * M * (c[1] + c[2]))
    sy = 2 * s[1] * (N + 2 * M * (c[0] + c[2]))
    sz = 2 * s[2] * (N + 2 * M * (c[0] + c[1]))
    lam = (2 * Q * (c[0] + c[1] + c[2]) + 4 * R * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2])
           - (6 * Q + 12 * R))
    return (sx, sy, sz), lam


@pytest.mark.parametrize("dims", [2, 3])
def test_stencil_fourier_symbols(dims):
    rng = np.random.default_rng(1)
    for N, Q in [(0.5, 1.0), (0.3, 2.5), (0.2, 0.4)]:
        if dims == 2:
            p = _params(2, 12, 10, N=N, Q=Q)
        else:
            p = _params(3, 6, 8, 10, N=N, Q=Q)
        L = np.array([p.Lx, p.Ly, p.Lz][:dims], dtype=float)
        coords = _coords(p)
        for _ in range(4):
            kk = 2 * np.pi * rng.integers(0, 5, size=dims) / L
            phase = sum(kk[a] * coords[a] for a in range(dims))
            cosf = np.cos(phase)
            sig, lam = _fourier_symbols(dims, N, Q, kk)
            np.testing.assert_allclose(O.lap_D(p, cosf), lam * cosf, atol=1e-12)
            g = O.grad_D(p, cosf)
            for a in range(dims):
                np.testing.assert_allclose(g[a], -sig[a] * np.sin(phase), atol=1e-12)
            # standard Laplacian of the FD step: Q = 1, R = 0
            _, lam_std = _fourier_symbols(dims, 0.5, 1.0, kk)
            np.testing.assert_allclose(O.lap_std(p, cosf), lam_std * cosf, atol=1e-12)


# ---- c2/c3: equilibrium and forcing moments ------------------------------------------

@pytest.mark.parametrize("dims", [2, 3])
def test_equilibrium_moments(dims):
    """Eqs. 13-16: sum feq = n, sum feq e = n u, sum feq ee = n cs2 I + n u u."""
    e, w = O.lattice(dims)
    e = e[:, :dims].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    rng = np.random.default_rng(2)
    for _ in range(10):
        n = 0.8 + 0.4 * rng.random()
        u = 0.1 * (rng.random(dims) - 0.5)
        f = O.feq(dims, n, u)
        np.testing.assert_allclose(f.sum(), n, rtol=1e-15)
        np.testing.assert_allclose(f @ e, n * u, atol=1e-16)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, e, e),
                                   n / 3 * np.eye(dims) + n * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("dims", [2, 3])
def test_forcing_moments(dims):
    """Eqs. 20 and 26: sum Fi = A = 0, sum Fi e = B = (1 - 1/2tau) F,
    sum Fi ee = cs2 A I + (C + C^T)/2 with C = (1 - 1/2tau)(u F + F u)."""
    e, _ = O.lattice(dims)
    e = e[:, :dims].astype(float)
    rng = np.random.default_rng(3)
    for tau in [0.6, 1.0, 5.0]:
        pref = 1 - 1 / (2 * tau)
        for _ in range(5):
            u = 0.1 * (rng.random(dims) - 0.5)
            F = 1e-3 * (rng.random(dims) - 0.5)
            Fi = O.forcing_term(dims, tau, u, F)
            assert abs(Fi.sum()) < 1e-18
            np.testing.assert_allclose(Fi @ e, pref * F, atol=1e-18)
            C = pref * (np.outer(u, F) + np.outer(F, u))
            np.testing.assert_allclose(np.einsum("i,ia,ib->ab", Fi, e, e), C, atol=1e-18)


def test_lattice_isotropy():
    """Lattice tensors of Sec. II A: sum w e e = cs2 I and sum w e e e e =
    cs2^2 (delta delta + delta delta + delta delta) for D2Q9 and D3Q19."""
    for dims in (2, 3):
        e, w = O.lattice(dims)
        e = e[:, :dims].astype(float)
        I = np.eye(dims)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, e, e), I / 3, atol=1e-16)
        four = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
        want = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                + np.einsum("ad,bc->abcd", I, I)) / 9
        np.testing.assert_allclose(four, want, atol=1e-16)
        # opposite directions pair up
        for i in range(len(w)):
            assert any(np.all(e[j] == -e[i]) for j in range(len(w)))


# ---- c9: FD operators through exact amplification factors (Eqs. 32-36) -------------

@pytest.mark.parametrize("dims", [2, 3])
def test_diffusion_linear_mode(dims):
    """u = 0, phi = pbar + eps cos(k.r): one substep multiplies the mode by
    1 - dt Gamma (a_eff lam + kappa lam^2), a_eff = a + 3 b pbar^2, with lam the
    symbol of the 5-point (7-point) Laplacian."""
    if dims == 2:
        p = _params(2, 16, 12, a=-0.1, b=0.1, kappa=0.14, Gamma=0.5, m=4)
    else:
        p = _params(3, 8, 6, 10, a=-0.1, b=0.1, kappa=0.14, Gamma=0.5, m=8)
    coords = _coords(p)
    L = np.array([p.Lx, p.Ly, p.Lz][:dims], dtype=float)
    u = np.zeros((dims,) + p.shape)
    for pbar in [0.0, 0.5, -0.9]:
        for kidx in [(1, 0, 0), (2, 3, 1), (4, 1, 2)]:
            kk = 2 * np.pi * np.array(kidx[:dims]) / L
            phase = sum(kk[a] * coords[a] for a in range(dims))
            eps = 1e-7
            phi = pbar + eps * np.cos(phase)
            dt = 1 / p.m
            half = O.advect(p, phi, u, dt)
            assert np.array_equal(half, phi)
            out = O.diffuse(p, half, phi, dt)
            lam = -sum(4 * np.sin(k / 2) ** 2 for k in kk)
            aeff = p.a + 3 * p.b * pbar ** 2
            G = 1 + dt * p.Gamma * (aeff * lam - p.kappa * lam * lam)
            amp = np.sum((out - pbar) * np.cos(phase)) / np.sum(np.cos(phase) ** 2)
            np.testing.assert_allclose(amp / eps, G, rtol=2e-6, atol=1e-9)


def test_advection_amplification_factors():
    """Constant u: the upwind step multiplies exp(ikx) by 1 - dt U (1 - e^{-ik})
    for U > 0 and by 1 - dt U (e^{ik} - 1) for U < 0 (Eqs. 32, 34, 35); uniform
    phi with u = U sin(kx) gives phi (1 - dt U sin k cos kx) (Eqs. 32, 33)."""
    p = _params(2, 16, 8)
    x, y = _coords(p)
    k = 2 * np.pi * 3 / 16
    dt = 0.25
    for U in (0.05, -0.07):
        u = np.zeros((2,) + p.shape)
        u[0] = U
        phi = np.cos(k * x)
        out = O.advect(p, phi, u, dt)
        G = 1 - dt * U * (1 - np.exp(-1j * k)) if U > 0 else 1 - dt * U * (np.exp(1j * k) - 1)
        np.testing.assert_allclose(out, np.real(G * np.exp(1j * k * x)), atol=1e-15)
        # y direction, same rule
        u = np.zeros((2,) + p.shape)
        u[1] = U
        phi = np.cos(2 * np.pi * y / 8)
        ky = 2 * np.pi / 8
        G = 1 - dt * U * (1 - np.exp(-1j * ky)) if U > 0 else 1 - dt * U * (np.exp(1j * ky) - 1)
        np.testing.assert_allclose(O.advect(p, phi, u, dt), np.real(G * np.exp(1j * ky * y)),
                                   atol=1e-15)
    u = np.zeros((2,) + p.shape)
    U = 0.03
    u[0] = U * np.sin(k * x)
    phi = np.full(p.shape, 0.8)
    np.testing.assert_allclose(O.advect(p, phi, u, dt),
                               0.8 * (1 - dt * U * np.sin(k) * np.cos(k * x)), atol=1e-15)


def test_advection_sum_by_parts():
    """Sum over a periodic grid of the printed advection step (Eqs. 32-35):
    sum phi' = sum phi + dt sum_alpha |u_alpha| (phi_+ - 2 phi + phi_-)/2
    (summation by parts); the flux form conserves sum phi exactly."""
    rng = np.random.default_rng(4)
    for dims, shape in [(2, (9, 13)), (3, (5, 6, 7))]:
        if dims == 2:
            p = _params(2, shape[1], shape[0])
        else:
            p = _params(3, shape[2], shape[1], shape[0])
        phi = rng.random(p.shape) - 0.5
        u = 0.1 * (rng.random((dims,) + p.shape) - 0.5)
        u[0].flat[::5] = 0.0  # exercise the u = 0 tie
        dt = 0.3
        out = O.advect(p, phi, u, dt)
        ax = {0: -1, 1: -2, 2: -3}
        drift = 0.0
        for a in range(dims):
            d2 = np.roll(phi, -1, ax[a]) - 2 * phi + np.roll(phi, 1, ax[a])
            drift += np.sum(np.abs(u[a]) * d2) / 2
        np.testing.assert_allclose(out.sum() - phi.sum(), dt * drift, atol=1e-13)
        pf = O.Params(**{**p.__dict__, "adv_variant": 1})
        outf = O.advect(pf, phi, u, dt)
        assert abs(outf.sum() - phi.sum()) < 1e-13
        # diffusion conserves sum phi in both variants
        dd = O.diffuse(p, out, phi, dt)
        assert abs(dd.sum() - out.sum()) < 1e-12


# ---- c11: brute force on tiny periodic grids ---------------------------------------

def _shift_matrix(shape, d):
    """Dense matrix P with (P v)[r] = v[r + d] on a periodic grid (numpy axes
    order [z][y][x]; d given as (dx, dy[, dz]))."""
    S = int(np.prod(shape))
    I = np.eye(S).reshape((S,) + tuple(shape))
    axes = tuple(range(1, len(shape) + 1))[::-1]
    # row k of the rolled identity is the one-hot field at site k moved by -d,
    # i.e. entry [k, r] = [k == r + d]; its transpose picks v[r + d] in row r.
    return np.roll(I, shift=tuple(-x for x in d), axis=axes).reshape(S, S).T


def _stencil_matrices_2d(shape, N, Q):
    """Dense d_Dx, d_Dy, lap_D from the printed 3x3 matrices (Eqs. 30-31)."""
    M = (1 - 2 * N) / 4
    R = (1 - Q) / 2
    dx_mat = np.array([[-M, 0, M], [-N, 0, N], [-M, 0, M]])
    lap_mat = np.array([[R, Q, R], [Q, -4 * (Q + R), Q], [R, Q, R]])
    S = int(np.prod(shape))
    Dx = np.zeros((S, S))
    Dy = np.zeros((S, S))
    Lp = np.zeros((S, S))
    for row in range(3):
        for col in range(3):
            d = (col - 1, row - 1)  # the matrix is symmetric in its rows
            P = _shift_matrix(shape, d)
            Dx += dx_mat[row, col] * P
            Dy += dx_mat.T[row, col] * P
            Lp += lap_mat[row, col] * P
    return Dx, Dy, Lp


def _stencil_matrices_3d(shape, N, Q):
    """Dense d_D and lap_D on the D3Q19 neighbourhood (3D generalisation of
    Eqs. 30-31: N/M on faces/edges with e_alpha != 0, Q/R on faces/edges)."""
    M = (1 - 2 * N) / 8
    R = (1 - Q) / 4
    S = int(np.prod(shape))
    D = [np.zeros((S, S)) for _ in range(3)]
    Lp = -(6 * Q + 12 * R) * np.eye(S)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nn = dx * dx + dy * dy + dz * dz
                if nn not in (1, 2):
                    continue
                P = _shift_matrix(shape, (dx, dy, dz))
                Lp += (Q if nn == 1 else R) * P
                for a, da in enumerate((dx, dy, dz)):
                    D[a] += (N if nn == 1 else M) * da * P
    return D, Lp


def _check_full_step(p, shape, D, Lp, L5, rng):
    """Force, collision, streaming and one FD substep of the oracle against
    dense operators; per-site feq / forcing come from the moment-pinned
    oracle functions."""
    dims = p.dims
    S = int(np.prod(shape))
    phi = 0.9 * (rng.random(shape) - 0.5)
    v = phi.reshape(-1)
    g = O.grad_D(p, phi)
    for a in range(dims):
        np.testing.assert_allclose(g[a].reshape(-1), D[a] @ v, atol=1e-14)
    np.testing.assert_allclose(O.lap_D(p, phi).reshape(-1), Lp @ v, atol=1e-14)
    np.testing.assert_allclose(O.lap_std(p, phi).reshape(-1), L5 @ v, atol=1e-14)
    mu = p.a * v + p.b * v ** 3 - p.kappa * (Lp @ v)
    np.testing.assert_allclose(O.mu(p, phi).reshape(-1), mu, atol=1e-14)
    n = 1 + 0.01 * (rng.random(shape) - 0.5)
    nv = n.reshape(-1)
    F_on = O.force(p, phi, n, t=0)
    F_off = O.force(p, phi, n, t=p.force_steps)
    for a in range(dims):
        np.testing.assert_allclose(F_on[a].reshape(-1), -v * (D[a] @ mu) + nv * p.g[a], atol=1e-14)
        np.testing.assert_allclose(F_off[a].reshape(-1), -v * (D[a] @ mu), atol=1e-14)
    e, w = O.lattice(dims)
    q = len(w)
    u0 = 0.01 * (rng.random((dims,) + shape) - 0.5)
    f = O.init(p, n, phi, u0)
    fv = f.reshape(q, -1)
    dens = fv.sum(0)
    np.testing.assert_allclose(dens, nv, rtol=1e-14)
    F = O.force(p, phi, dens.reshape(shape), t=0)
    Fv = F.reshape(dims, -1)
    u = np.stack([((fv * e[:, a:a + 1]).sum(0) + Fv[a] / 2) / dens for a in range(dims)])
    np.testing.assert_allclose(u, u0.reshape(dims, -1), atol=1e-15)
    post = np.zeros_like(fv)
    for s in range(S):
        feq = O.feq(dims, dens[s], u[:, s])
        Fi = O.forcing_term(dims, p.tau, u[:, s], Fv[:, s])
        post[:, s] = fv[:, s] - (fv[:, s] - feq) / p.tau + Fi
    streamed = np.stack([_shift_matrix(shape, tuple(-int(x) for x in e[i, :dims])) @ post[i]
                         for i in range(q)])
    f2 = f.copy()
    n_t, u_t = O.lb_step(p, f2, phi, 0)
    np.testing.assert_allclose(f2.reshape(q, -1), streamed, atol=1e-15)
    np.testing.assert_allclose(u_t.reshape(dims, -1), u, atol=1e-15)
    dt = 1 / p.m
    I = np.eye(S)
    half = v.copy()
    tend = np.zeros(S)
    for a in range(dims):
        unit = [0, 0, 0][:dims]
        unit[a] = 1
        Pp = _shift_matrix(shape, tuple(unit))
        Pm = _shift_matrix(shape, tuple(-x for x in unit))
        ua = u_t[a].reshape(-1)
        dphi = np.where(ua < 0, (Pp - I) @ v, (I - Pm) @ v)
        tend += v * (((Pp - Pm) / 2) @ ua) + ua * dphi
    half = v - dt * tend
    np.testing.assert_allclose(O.advect(p, phi, u_t, dt).reshape(-1), half, atol=1e-15)
    new = half + dt * p.Gamma * (p.a * (L5 @ half) + p.b * (L5 @ v ** 3)
                                 - p.kappa * (L5 @ (L5 @ half)))
    np.testing.assert_allclose(O.diffuse(p, half.reshape(shape), phi, dt).reshape(-1), new,
                               atol=1e-14)


@pytest.mark.parametrize("shape", [(3, 3), (5, 4), (2, 3), (4, 7)])
def test_bruteforce_tiny_2d(shape):
    """Stencils rebuilt as dense matrices from the printed 3x3 matrices
    (Eqs. 30-31), streaming as permutations, one full hybrid step."""
    Ly, Lx = shape
    rng = np.random.default_rng(5)
    p = _params(2, Lx, Ly, N=0.3, Q=2.5, a=-0.1, b=0.1, kappa=0.14, tau=0.9, Gamma=0.5, m=3,
                g=(1e-4, -2e-4, 0.0), force_steps=5)
    Dx, Dy, Lp = _stencil_matrices_2d(shape, p.N, p.Q)
    _, _, L5 = _stencil_matrices_2d(shape, 0.5, 1.0)
    _check_full_step(p, shape, [Dx, Dy], Lp, L5, rng)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 3)])
def test_bruteforce_tiny_3d(shape):
    """The same on D3Q19 tiny periodic grids."""
    rng = np.random.default_rng(6)
    Lz, Ly, Lx = shape
    p = _params(3, Lx, Ly, Lz, N=0.3, Q=0.5, a=-0.1, b=0.1, kappa=0.14, tau=1.3, Gamma=0.5,
                m=2, g=(1e-4, 2e-4, -1e-4), force_steps=3)
    D, Lp = _stencil_matrices_3d(shape, p.N, p.Q)
    _, L7 = _stencil_matrices_3d(shape, 0.5, 1.0)
    _check_full_step(p, shape, D, Lp, L7, rng)
