"""Host-side model of the fused 3D FD kernel (csrc/kernels_3d.cu, fd3g_kernel:
the advection of Eqs. 32-35 and both halves of Eq. 36 in one z-marching
kernel), run on the CPU against the oracle's FD substep.

The model follows the kernel's grid (F3G_NW-warp CTAs owning F3G_NW - 4
output rows, z chunks sized as the host sizes them), each warp's row and
wrapped neighbours, its registers (phih of planes k, k + 1, k + 2) and the two
shared-memory rings (phih: two planes, psi: four), with every ring entry
tagged by the plane it holds.  Between two barriers the warps run in any
order, so within one such segment no ring entry may be both read and
written; every read must find the plane the arithmetic needs; every output
site must be written exactly once; and the result must equal one FD substep
of the oracle (advect then diffuse)."""
import numpy as np
import pytest

import oracle as O

NW = 16  # F3G_NW


def grid_of(Ly, Lz):
    rows_g = (Ly + NW - 5) // (NW - 4)
    zch = max(1, min(Lz, 152 // rows_g))
    nzg = max(min(8, Lz), (Lz + zch - 1) // zch)
    return rows_g, nzg, (Lz + nzg - 1) // nzg


class Segments:
    """Ring entries (ring, slot, warp) -> (plane, row); writes become visible
    at the next barrier, and a segment may not read and write one entry."""

    def __init__(self):
        self.store, self.pending, self.reads = {}, {}, set()

    def rd(self, key, plane):
        assert key not in self.pending, ("read and written in one segment", key)
        tag, row = self.store[key]
        assert tag == plane, ("stale ring entry", key, tag, plane)
        self.reads.add(key)
        return row

    def wr(self, key, plane, row):
        assert key not in self.reads and key not in self.pending, ("race", key)
        self.pending[key] = (plane, row)

    def barrier(self):
        self.store.update(self.pending)
        self.pending, self.reads = {}, set()


def adv_row(phi, u, y, zz, dt, flux):
    """phih of row y on plane zz, whole rows (x periodic)."""
    Lz, Ly, _ = phi.shape
    z, zm, zp, ym, yp = zz % Lz, (zz - 1) % Lz, (zz + 1) % Lz, (y - 1) % Ly, (y + 1) % Ly
    ph = phi[z, y]

    def term(fm, fp, cm, c, cp):
        if not flux:
            return ph * ((cp - cm) / 2) + c * np.where(c < 0, fp - ph, ph - fm)
        Up, Um = 0.5 * (c + cp), 0.5 * (cm + c)
        return np.where(Up > 0, Up * ph, Up * fp) - np.where(Um > 0, Um * fm, Um * ph)

    U, V, Wv = u[0], u[1], u[2]
    tend = term(np.roll(ph, 1), np.roll(ph, -1), np.roll(U[z, y], 1), U[z, y], np.roll(U[z, y], -1))
    tend = tend + term(phi[z, ym], phi[z, yp], V[z, ym], V[z, y], V[z, yp])
    tend = tend + term(phi[zm, y], phi[zp, y], Wv[zm, y], Wv[z, y], Wv[zp, y])
    return ph - dt * tend


def lap_row(c, m, p, ym, yp):
    return m + p + ym + yp + np.roll(c, 1) + np.roll(c, -1) - 6 * c


def fd3g_model(phi, u, p, dt, flux=False, cubic_half=False):
    Lz, Ly, Lx = phi.shape
    out = np.full(phi.shape, np.nan)
    rows_g, nzg, chunks = grid_of(Ly, Lz)
    dtG = dt * p.Gamma
    for by in range(rows_g):
        for bz in range(chunks):
            y0, z0 = by * (NW - 4), bz * nzg
            z1 = min(z0 + nzg, Lz)
            yr = [y0 - 2 + w for w in range(NW)]
            yw = [r % Ly for r in yr]
            psiw = [1 <= w <= NW - 2 for w in range(NW)]
            outw = [2 <= w <= NW - 3 and yr[w] < Ly for w in range(NW)]
            seg = Segments()
            hm = [adv_row(phi, u, yw[w], z0 - 2, dt, flux) for w in range(NW)]
            hc = [adv_row(phi, u, yw[w], z0 - 1, dt, flux) for w in range(NW)]
            hp = [None] * NW
            for w in range(NW):
                seg.wr(("h", (z0 - 1) & 1, w), z0 - 1, hc[w])
            for k in range(z0 - 2, z1):
                for w in range(NW):  # advection of plane k + 2
                    hp[w] = adv_row(phi, u, yw[w], k + 2, dt, flux)
                    seg.wr(("h", (k + 2) & 1, w), k + 2, hp[w])
                seg.barrier()
                for w in range(NW):  # psi of plane k + 1
                    if not psiw[w]:
                        continue
                    hym = seg.rd(("h", (k + 1) & 1, w - 1), k + 1)
                    hyp = seg.rd(("h", (k + 1) & 1, w + 1), k + 1)
                    cb = hc[w] if cubic_half else phi[(k + 1) % Lz, yw[w]]
                    psi = p.a * hc[w] + p.b * cb ** 3 - p.kappa * lap_row(hc[w], hm[w], hp[w], hym, hyp)
                    seg.wr(("q", (k + 1) & 3, w), k + 1, psi)
                seg.barrier()
                for w in range(NW):  # phi^{n+1} of plane k
                    if k >= z0 and outw[w]:
                        qc = seg.rd(("q", k & 3, w), k)
                        qm = seg.rd(("q", (k + 3) & 3, w), k - 1)
                        qp = seg.rd(("q", (k + 1) & 3, w), k + 1)
                        qym = seg.rd(("q", k & 3, w - 1), k)
                        qyp = seg.rd(("q", k & 3, w + 1), k)
                        assert np.all(np.isnan(out[k, yr[w]])), ("written twice", k, yr[w])
                        out[k, yr[w]] = hm[w] + dtG * lap_row(qc, qm, qp, qym, qyp)
                    hm[w], hc[w] = hc[w], hp[w]
            seg.barrier()
    return out


@pytest.mark.parametrize("shape", [(13, 9, 128), (21, 19, 256), (10, 30, 128), (5, 3, 256), (40, 26, 128)])
@pytest.mark.parametrize("flux", [False, True])
def test_fd3g_model_equals_oracle_substep(shape, flux):
    Lz, Ly, Lx = shape
    rng = np.random.default_rng(sum(shape) + flux)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((3,) + shape)
    u[:, ::3, ::2, ::5] = 0.0  # u = 0 takes the kernel's else branches
    p = O.Params(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, m=8, adv_variant=int(flux), N=1 / 6, Q=1 / 3)
    dt = 1.0 / p.m
    got = fd3g_model(phi, u, p, dt, flux=flux)
    assert not np.any(np.isnan(got))
    ref = O.diffuse(p, O.advect(p, phi, u, dt), phi, dt)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_fd3g_model_cubic_at_half():
    shape = (9, 14, 128)
    rng = np.random.default_rng(7)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((3,) + shape)
    p = O.Params(dims=3, Lx=128, Ly=14, Lz=9, m=4, cubic_at_half=1, N=1 / 6, Q=1 / 3)
    got = fd3g_model(phi, u, p, 0.25, cubic_half=True)
    ref = O.diffuse(p, O.advect(p, phi, u, 0.25), phi, 0.25)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_fd3g_grid_fits_one_wave():
    """One CTA per SM: the grid of the 256^3 and 128^3 lattices stays within
    the 152 SMs, and every chunk holds at least 8 planes (or the lattice)."""
    for Ly, Lz in ((256, 256), (128, 128), (96, 200), (9, 13)):
        rows_g, nzg, chunks = grid_of(Ly, Lz)
        assert rows_g * chunks <= 152 or chunks == 1
        assert nzg >= min(8, Lz) and (chunks - 1) * nzg < Lz <= chunks * nzg
