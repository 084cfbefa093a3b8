"""Host-side model of the pipelined 3D FD substep kernel (csrc/kernels_3d.cu,
fd3p_kernel: the advection of Eqs. 32-35 and both halves of Eq. 36 in one
z-marching kernel with one barrier per plane), run on the CPU against the
oracle's FD substep.

The model follows the kernel's grid (F3P_NW-warp CTAs owning F3P_NW - 4
output rows, z chunks sized as the host sizes them for 152 resident CTAs),
each warp's row and wrapped neighbours, its registers (own-row phi and w
of three planes marching in z, phi of rows y -+ 1, the cube's phi), the
shared-memory rings (phih: four slots, psi: three, u and v rows: two, filled
by bulk copies that complete on one mbarrier a slot), and the order of the
three phases within an iteration (C, B, A).  Every ring entry is tagged by
the plane it holds.  Between two barriers the warps run in any order, so an
entry one warp writes may not be touched by another warp in that segment;
the writing warp may read its own entry before it writes it (program
order).  Every read must find the plane the arithmetic needs, every copy
wait must use the parity of its completion, every output site must be
written exactly once, and the result must equal one FD substep of the
oracle (advect then diffuse)."""
import numpy as np
import pytest

import oracle as O

NW = 16  # F3P_NW
RESIDENT = 152


def grid_of(Ly, Lz, resident=RESIDENT):
    rows_p = (Ly + NW - 5) // (NW - 4)
    zch = max(1, min(Lz, resident // rows_p))
    nzp = (Lz + zch - 1) // zch
    return rows_p, nzp, (Lz + nzp - 1) // nzp


class Segments:
    """Ring entries -> (plane, row).  Writes become visible at the next
    barrier; within a segment an entry written by one warp may be read by
    no other warp, and an entry read by another warp may not be written."""

    def __init__(self):
        self.store, self.pending, self.readers = {}, {}, {}

    def rd(self, key, plane, warp):
        assert key not in self.pending, ("read after a write in one segment", key)
        tag, row = self.store[key]
        assert tag == plane, ("stale ring entry", key, tag, plane)
        self.readers.setdefault(key, set()).add(warp)
        return row

    def wr(self, key, plane, row, warp):
        assert self.readers.get(key, set()) <= {warp}, ("race", key, self.readers[key], warp)
        assert key not in self.pending, ("written twice in one segment", key)
        self.pending[key] = (plane, row)

    def barrier(self):
        self.store.update(self.pending)
        self.pending, self.readers = {}, {}


class CopyRing:
    """The two u/v slots: copies in flight per slot, completed in order; a
    wait names the parity of the completion it expects."""

    def __init__(self):
        self.issued = {0: [], 1: []}  # planes per slot, in issue order
        self.data = {}
        self.readers = {0: set(), 1: set()}

    def issue(self, pl, u, v, Ly, Lz, y0):
        s = pl & 1
        assert not self.readers[s], ("copy into a slot read in this segment", pl)
        self.issued[s].append(pl)
        z = pl % Lz
        self.data[(s, pl)] = ([u[z, (y0 - 2 + i) % Ly] for i in range(NW)],
                              [v[z, (y0 - 3 + i) % Ly] for i in range(NW + 2)])

    def wait(self, pl, parity):
        s = pl & 1
        n = self.issued[s].index(pl)
        assert n & 1 == parity, ("wrong parity", pl, n, parity)
        assert self.issued[s][-1] == pl, ("a later copy into the slot was issued before this one was read", pl)
        return self.data[(s, pl)]

    def read(self, pl, warp):
        self.readers[pl & 1].add(warp)

    def barrier(self):
        self.readers = {0: set(), 1: set()}


def adv_row(phi, u, y, zz, dt, flux, U_row=None, V_rows=None):
    """phih of row y on plane zz, whole rows (x periodic); u and v rows from
    the staged copies when given."""
    Lz, Ly, _ = phi.shape
    z, zm, zp, ym, yp = zz % Lz, (zz - 1) % Lz, (zz + 1) % Lz, (y - 1) % Ly, (y + 1) % Ly
    ph = phi[z, y]

    def term(fm, fp, cm, c, cp):
        if not flux:
            return ph * ((cp - cm) / 2) + c * np.where(c < 0, fp - ph, ph - fm)
        Up, Um = 0.5 * (c + cp), 0.5 * (cm + c)
        return np.where(Up > 0, Up * ph, Up * fp) - np.where(Um > 0, Um * fm, Um * ph)

    Uc = u[0][z, y] if U_row is None else U_row
    Vm, Vc, Vp = (u[1][z, ym], u[1][z, y], u[1][z, yp]) if V_rows is None else V_rows
    Wv = u[2]
    tend = term(np.roll(ph, 1), np.roll(ph, -1), np.roll(Uc, 1), Uc, np.roll(Uc, -1))
    tend = tend + term(phi[z, ym], phi[z, yp], Vm, Vc, Vp)
    tend = tend + term(phi[zm, y], phi[zp, y], Wv[zm, y], Wv[z, y], Wv[zp, y])
    return ph - dt * tend


def lap_row(c, m, p, ym, yp):
    return m + p + ym + yp + np.roll(c, 1) + np.roll(c, -1) - 6 * c


def fd3p_model(phi, u, p, dt, flux=False, cubic_half=False, resident=RESIDENT):
    Lz, Ly, Lx = phi.shape
    out = np.full(phi.shape, np.nan)
    rows_p, nzp, chunks = grid_of(Ly, Lz, resident)
    dtG = dt * p.Gamma
    for by in range(rows_p):
        for bz in range(chunks):
            y0, z0 = by * (NW - 4), bz * nzp
            z1 = min(z0 + nzp, Lz)
            a0, a1 = z0 - 2, z1 + 1
            yr = [y0 - 2 + w for w in range(NW)]
            yw = [r % Ly for r in yr]
            psiw = [1 <= w <= NW - 2 for w in range(NW)]
            outw = [2 <= w <= NW - 3 and yr[w] < Ly for w in range(NW)]
            seg, cp = Segments(), CopyRing()
            cp.issue(a0, u[0], u[1], Ly, Lz, y0)
            if a0 + 1 <= a1:
                cp.issue(a0 + 1, u[0], u[1], Ly, Lz, y0)
            # registers: own-row phi planes (a - 1, a, a + 1) as plane numbers,
            # the cube's plane; the values are read from phi by plane number
            reg = [{"P": [a0 - 1, a0, a0 + 1], "Pk": None} for _ in range(NW)]
            for k in range(z0 - 4, z1 + 2):
                if k >= z0 - 3 and k + 3 <= a1:
                    cp.issue(k + 3, u[0], u[1], Ly, Lz, y0)
                for w in range(NW):
                    # C: phi^{n+1} of plane k - 2
                    if k >= z0 + 2 and outw[w]:
                        zc = k - 2
                        qc = seg.rd(("q", (zc + 6) % 3, w), zc, w)
                        qm = seg.rd(("q", (zc + 5) % 3, w), zc - 1, w)
                        qp = seg.rd(("q", (zc + 7) % 3, w), zc + 1, w)
                        qym = seg.rd(("q", (zc + 6) % 3, w - 1), zc, w)
                        qyp = seg.rd(("q", (zc + 6) % 3, w + 1), zc, w)
                        hm = seg.rd(("h", zc & 3, w), zc, w)
                        assert np.all(np.isnan(out[zc, yr[w]])), ("written twice", zc, yr[w])
                        out[zc, yr[w]] = hm + dtG * lap_row(qc, qm, qp, qym, qyp)
                    # B: psi of plane k
                    if z0 - 1 <= k <= z1 and psiw[w]:
                        hc = seg.rd(("h", k & 3, w), k, w)
                        hm = seg.rd(("h", (k + 3) & 3, w), k - 1, w)
                        hp = seg.rd(("h", (k + 1) & 3, w), k + 1, w)
                        hym = seg.rd(("h", k & 3, w - 1), k, w)
                        hyp = seg.rd(("h", k & 3, w + 1), k, w)
                        assert reg[w]["Pk"] == k, ("cube from the wrong plane", reg[w]["Pk"], k)
                        cb = hc if cubic_half else phi[k % Lz, yw[w]]
                        psi = p.a * hc + p.b * cb ** 3 - p.kappa * lap_row(hc, hm, hp, hym, hyp)
                        seg.wr(("q", (k + 6) % 3, w), k, psi, w)
                    # A: phih of plane k + 2
                    a = k + 2
                    r = reg[w]
                    if a <= a1:
                        assert r["P"] == [a - 1, a, a + 1], ("marching registers", r["P"], a)
                        U, V = cp.wait(a, ((a - a0) >> 1) & 1)
                        cp.read(a, w)
                        h = adv_row(phi, u, yw[w], a, dt, flux, U_row=U[w], V_rows=(V[w], V[w + 1], V[w + 2]))
                        seg.wr(("h", a & 3, w), a, h, w)
                        r["Pk"] = r["P"][0]
                        r["P"] = [a, a + 1, a + 2]
                    else:
                        r["Pk"] = r["P"][0]
                        r["P"] = [r["P"][1], r["P"][2], None]
                seg.barrier()
                cp.barrier()
    return out


@pytest.mark.parametrize("shape", [(13, 9, 128), (21, 19, 256), (10, 30, 128), (5, 3, 256), (40, 26, 128)])
@pytest.mark.parametrize("flux", [False, True])
def test_fd3p_model_equals_oracle_substep(shape, flux):
    Lz, Ly, Lx = shape
    rng = np.random.default_rng(sum(shape) + flux)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((3,) + shape)
    u[:, ::3, ::2, ::5] = 0.0  # u = 0 takes the kernel's else branches
    p = O.Params(dims=3, Lx=Lx, Ly=Ly, Lz=Lz, m=8, adv_variant=int(flux), N=1 / 6, Q=1 / 3)
    dt = 1.0 / p.m
    got = fd3p_model(phi, u, p, dt, flux=flux)
    assert not np.any(np.isnan(got))
    ref = O.diffuse(p, O.advect(p, phi, u, dt), phi, dt)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("resident", [152, 304, 7])
def test_fd3p_model_other_chunkings(resident):
    """Chunk heights of one plane (many CTAs) up to the whole lattice."""
    shape = (11, 14, 128)
    rng = np.random.default_rng(resident)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((3,) + shape)
    p = O.Params(dims=3, Lx=128, Ly=14, Lz=11, m=8, N=1 / 6, Q=1 / 3)
    got = fd3p_model(phi, u, p, 0.125, resident=resident)
    ref = O.diffuse(p, O.advect(p, phi, u, 0.125), phi, 0.125)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_fd3p_model_cubic_at_half():
    shape = (9, 14, 128)
    rng = np.random.default_rng(7)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((3,) + shape)
    p = O.Params(dims=3, Lx=128, Ly=14, Lz=9, m=4, cubic_at_half=1, N=1 / 6, Q=1 / 3)
    got = fd3p_model(phi, u, p, 0.25, cubic_half=True)
    ref = O.diffuse(p, O.advect(p, phi, u, 0.25), phi, 0.25)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_fd3p_grid_fits_one_wave():
    """One CTA per SM: the grid of the 256^3 and 128^3 lattices stays within
    the 152 SMs."""
    for Ly, Lz in ((256, 256), (128, 128), (96, 200), (9, 13)):
        rows_p, nzp, chunks = grid_of(Ly, Lz)
        assert rows_p * chunks <= 152 or chunks == 1
        assert (chunks - 1) * nzp < Lz <= chunks * nzp
