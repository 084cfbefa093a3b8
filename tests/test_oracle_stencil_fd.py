"""Pins of the oracle's stencil_fd option: the stencil operators of Eqs. 30-31
(at the force's N, Q) in place of the central d u of Eq. 33 and the 5-point
Laplacian of Eq. 36 -- the "more general stencil" the paper mentions after
Eq. 36 (Sec. II C) and in Sec. IV.  Each pin is fixed by something other than
the oracle: the printed scheme it reduces to, or a Fourier closed form."""
import numpy as np
import pytest

import oracle as O


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((2,) + shape)
    return phi, u


def test_sc_stencil_is_the_printed_scheme_bitwise():
    """N = 1/2, Q = 1 (M = R = 0): the stencil operators are the central
    difference and the 5-point Laplacian, so both forms give the same bits."""
    shape = (23, 31)
    phi, u = _fields(shape, 1)
    kw = dict(Lx=31, Ly=23, N=0.5, Q=1.0, m=4)
    p0, p1 = O.Params(stencil_fd=0, **kw), O.Params(stencil_fd=1, **kw)
    a0, a1 = O.advect(p0, phi, u, 0.25), O.advect(p1, phi, u, 0.25)
    assert np.array_equal(a0, a1)
    assert np.array_equal(O.diffuse(p0, a0, phi, 0.25), O.diffuse(p1, a1, phi, 0.25))


@pytest.mark.parametrize("N,Q", [(0.3, 2.5), (7 / 12, 7 / 6), (1 / 3, 2 / 3)])
@pytest.mark.parametrize("nx,ny", [(1, 0), (2, 3), (5, 5), (7, 2)])
def test_diffusion_mode_factor_uses_the_stencil_laplacian(N, Q, nx, ny):
    """One diffusive substep on phi = eps cos(k.r) with u = 0 multiplies the
    mode by 1 - dt Gamma (a lam_D + kappa lam_D^2) (Eq. 36 linearised; the
    cube is O(eps^3)), lam_D = 4(Q + R) - 2Q (cos kx + cos ky) - 4R cos kx cos ky
    the symbol of -lap_D of Eq. 31 with R = (1 - Q)/2.  A 5-point Laplacian
    left in any of the three places changes the factor of diagonal modes."""
    Lx, Ly = 40, 36
    kx, ky = 2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly
    y, x = np.mgrid[0:Ly, 0:Lx]
    eps = 1e-7
    phi = eps * np.cos(kx * x + ky * y)
    p = O.Params(Lx=Lx, Ly=Ly, N=N, Q=Q, m=4, stencil_fd=1)
    dt = 0.25
    out = O.diffuse(p, phi, phi, dt)
    R = (1 - Q) / 2
    lam = 4 * (Q + R) - 2 * Q * (np.cos(kx) + np.cos(ky)) - 4 * R * np.cos(kx) * np.cos(ky)
    factor = 1 - dt * p.Gamma * (p.a * lam + p.kappa * lam ** 2)
    np.testing.assert_allclose(out, factor * phi, rtol=0, atol=1e-12 * eps)


@pytest.mark.parametrize("N", [0.3, 0.45, 7 / 12])
def test_advection_divergence_uses_the_stencil_derivative(N):
    """Uniform phi: the upwind terms vanish and phih = phi (1 - dt d_D.u*);
    for u*_x = U sin(kx x + ky y) the stencil derivative of Eq. 30 is
    U sin kx (2N + 4M cos ky) cos(kx x + ky y), M = (1 - 2N)/4 (and the same
    with x and y exchanged for u*_y)."""
    Lx, Ly = 32, 30
    y, x = np.mgrid[0:Ly, 0:Lx]
    kx, ky, px, py = 2 * np.pi * 3 / Lx, 2 * np.pi * 2 / Ly, 2 * np.pi * 5 / Lx, 2 * np.pi * 4 / Ly
    U, V = 0.01, 0.007
    u = np.stack([U * np.sin(kx * x + ky * y), V * np.sin(px * x + py * y)])
    phi = np.full((Ly, Lx), 0.7)
    M = (1 - 2 * N) / 4
    p = O.Params(Lx=Lx, Ly=Ly, N=N, Q=2.5, m=4, stencil_fd=1)
    dt = 0.25
    div = (U * np.sin(kx) * (2 * N + 4 * M * np.cos(ky)) * np.cos(kx * x + ky * y)
           + V * np.sin(py) * (2 * N + 4 * M * np.cos(px)) * np.cos(px * x + py * y))
    np.testing.assert_allclose(O.advect(p, phi, u, dt), 0.7 * (1 - dt * div), rtol=0, atol=1e-15)
    # the printed scheme's central difference is the N = 1/2 case
    p0 = O.Params(Lx=Lx, Ly=Ly, N=N, Q=2.5, m=4, stencil_fd=0)
    div0 = U * np.sin(kx) * np.cos(kx * x + ky * y) + V * np.sin(py) * np.cos(px * x + py * y)
    np.testing.assert_allclose(O.advect(p0, phi, u, dt), 0.7 * (1 - dt * div0), rtol=0, atol=1e-15)


def test_stencil_fd_step_brute_force_tiny_grid():
    """One full FD step (m substeps) on a 5 x 4 lattice against dense operator
    matrices built from the printed stencil matrices of Eqs. 30-31."""
    Lx, Ly = 5, 4
    N, Q = 0.3, 2.5
    M, R = (1 - 2 * N) / 4, (1 - Q) / 2
    S = Lx * Ly

    def idx(x, y):
        return (y % Ly) * Lx + (x % Lx)

    Dx, Dy, L = np.zeros((S, S)), np.zeros((S, S)), np.zeros((S, S))
    for y in range(Ly):
        for x in range(Lx):
            s = idx(x, y)
            for dx, dy, w in ((1, 0, N), (-1, 0, -N), (1, 1, M), (-1, 1, -M), (1, -1, M), (-1, -1, -M)):
                Dx[s, idx(x + dx, y + dy)] += w
                Dy[s, idx(x + dy, y + dx)] += w
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                L[s, idx(x + dx, y + dy)] += Q
            for dx, dy in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                L[s, idx(x + dx, y + dy)] += R
            L[s, s] += -4 * (Q + R)
    phi, u = _fields((Ly, Lx), 9)
    p = O.Params(Lx=Lx, Ly=Ly, N=N, Q=Q, m=2, stencil_fd=1)
    dt = 0.5
    f, ux, uy = phi.reshape(-1), u[0].reshape(-1), u[1].reshape(-1)
    for _ in range(p.m):
        up_x = np.where(ux < 0, np.roll(phi, -1, 1).reshape(-1) - f, f - np.roll(phi, 1, 1).reshape(-1))
        up_y = np.where(uy < 0, np.roll(phi, -1, 0).reshape(-1) - f, f - np.roll(phi, 1, 0).reshape(-1))
        h = f - dt * (f * (Dx @ ux + Dy @ uy) + ux * up_x + uy * up_y)
        f = h + dt * p.Gamma * (p.a * (L @ h) + p.b * (L @ f ** 3) - p.kappa * (L @ (L @ h)))
        phi = f.reshape(Ly, Lx)
    ref = np.ascontiguousarray(_fields((Ly, Lx), 9)[0])
    O.fd_step(p, ref, u)  # in place
    np.testing.assert_allclose(ref, phi, rtol=0, atol=1e-13)
