"""Host-side model of the y-marching 2D FD kernel (csrc/fd2d_wave.cu: SUB
substeps of Eqs. 32-36 per launch, warp A running substeps 1-2 and warp B
substeps 3-4), run on the CPU against the oracle's FD substeps.

The model follows the kernel's grid (128-column strips writing their inner
128 - 2 HX columns, segments of NY output rows reading HY = 3 SUB rows on
either side), its tick schedule (input row j lands at tick j; warp A works on
row a = t - 1, warp B on b = t - 9), the per-lane input rings (slot j % 8,
prefetched 6 rows ahead), the shared coefficient ring (slot r % 16 for four
substeps, r % 4 for two; warp A writes row t - 1 and reads row t - 4, warp B
reads rows t - 9 and t - 12) and the four-slot phi_2 hand-over, with one
barrier after every second tick.  Shuffles past the strip's edge read NaN, every ring slot starts
as NaN and keeps its last contents (the kernel computes through the fill and
drain ticks on whatever the slots hold), writes to the shared rings become
visible at the tick's barrier and may not touch a slot read in the same
tick, and every lattice site must be written exactly once with the oracle's
value."""
import numpy as np
import pytest

import oracle as O

W, IR, D = 128, 8, 6


def consts(sub):
    hy = 3 * sub
    hx = (3 * sub + 3) // 4 * 4
    lag = 14 if sub == 4 else 6
    return hy, hx, W - 2 * hx, lag


def ticks(sub, NY):
    hy, _, _, lag = consts(sub)
    return (NY + hy + lag + 1) // 2 * 2


def left(x):
    return np.concatenate(([np.nan], x[:-1]))


def right(x):
    return np.concatenate((x[1:], [np.nan]))


def coef(uc, vm, vc, vp, dt):
    div = (right(uc) - left(uc)) * 0.5 + (vp - vm) * 0.5
    return (1.0 - dt * (div + (np.abs(uc) + np.abs(vc))), dt * uc, dt * vc)


class Sub:
    """One substep's row windows: phi^n rows a-1, a; phih a-2, a-1; psi a-3, a-2."""

    def __init__(self):
        nan = np.full(W, np.nan)
        self.pm = self.pc = self.hu = self.hc = self.qu = self.qc = nan

    def step(self, pn, cf, p, dt, cubic_half):
        c0, t1, t2 = cf
        upx = np.where(t1 > 0, left(self.pc), right(self.pc))
        upy = np.where(t2 > 0, self.pm, pn)
        hn = c0 * self.pc + np.abs(t1) * upx + np.abs(t2) * upy
        cb = self.hc if cubic_half else self.pm
        lap = -4 * self.hc + ((self.hu + hn) + (left(self.hc) + right(self.hc)))
        qn = p.a * self.hc + (p.b * cb ** 3 + (-p.kappa) * lap)
        lapq = -4 * self.qc + ((self.qu + qn) + (left(self.qc) + right(self.qc)))
        out = p.Gamma * dt * lapq + self.hu
        self.pm, self.pc, self.hu, self.hc, self.qu, self.qc = self.pc, pn, self.hc, hn, self.qc, qn
        return out


def wave_model(phi, u, p, sub, NY, cubic_half=False, lag_b=14):
    Ly, Lx = phi.shape
    hy, hx, tx, lag = consts(sub)
    dt = 1.0 / p.m
    out = np.full(phi.shape, np.nan)
    nstrips, nsegs = (Lx + tx - 1) // tx, (Ly + NY - 1) // NY
    for bx in range(nstrips):
        x0 = bx * tx - hx
        cols = (x0 + np.arange(W)) % Lx
        wcols = np.arange(W)
        col_ok = (wcols >= hx) & (wcols < hx + tx) & (x0 + wcols < Lx)
        for by in range(nsegs):
            ys = by * NY
            J = NY + 2 * hy
            T = ticks(sub, NY)
            rings = {k: [(None, np.full(W, np.nan))] * IR for k in "puv"}
            CR = 16 if sub == 4 else 4
            coef_ring = [(None, (np.nan,) * 3)] * CR
            hand = [(None, np.full(W, np.nan))] * 4
            writes = {}
            sa1, sa2, sb1, sb2 = Sub(), Sub(), Sub(), Sub()
            vm = vc = np.full(W, np.nan)

            def issue(j):
                if j < J:
                    y = (ys - hy + j) % Ly
                    for k, src in (("p", phi[y]), ("u", u[0][y]), ("v", u[1][y])):
                        rings[k][j % IR] = (j, src[cols])

            def rd_in(k, j):
                tag, row = rings[k][j % IR]
                if 0 <= j < J:
                    assert tag == j, ("input ring", k, j, tag)
                return row

            for j in range(D):
                issue(j)
            for t in range(T):
                # ---- warp A ----
                issue(t + D)
                pn, vn, uc = rd_in("p", t), rd_in("v", t), rd_in("u", t - 1)
                cf = coef(uc, vm, vc, vn, dt)
                vm, vc = vc, vn
                # warp A's own ring entries are visible to it at once (each lane
                # reads back the columns it wrote); warp B sees them after the barrier
                coef_ring[(t - 1) % CR] = (t - 1, cf)
                o1 = sa1.step(pn, cf, p, dt, cubic_half)
                tag, cf2 = coef_ring[(t - 4) % CR]
                assert tag == t - 4 or t < 4, ("coefficient ring, warp A", t, tag)
                o2 = sa2.step(o1, cf2, p, dt, cubic_half)
                if t % 2 == 0:
                    written_c = set()  # slots written since the last barrier
                written_c.add((t - 1) % CR)
                if sub == 4:
                    writes[("h", (t - 6) % 4)] = (t - 6, o2)
                else:
                    r = t - 6
                    if hy <= r < hy + NY and ys + r - hy < Ly:
                        y = ys + r - hy
                        for cc in np.nonzero(col_ok)[0]:
                            assert np.isnan(out[y, x0 + cc]), ("written twice", y, x0 + cc)
                            out[y, x0 + cc] = o2[cc]
                # ---- warp B ----
                if sub == 4:
                    assert not ({(t - 9) % CR, (t - 12) % CR} & written_c), ("coefficient slot race", t)
                    assert ("h", (t - 8) % 4) not in writes, ("hand-over slot race", t)
                    htag, pnb = hand[(t - 8) % 4]
                    assert htag == t - 8 or t < 8, ("hand-over", t, htag)
                    ctag, cfb = coef_ring[(t - 9) % CR]
                    assert ctag == t - 9 or t < 10, ("coefficient ring, warp B", t, ctag)
                    o3 = sb1.step(pnb, cfb, p, dt, cubic_half)
                    ctag, cf4 = coef_ring[(t - 12) % CR]
                    assert ctag == t - 12 or t < 13, ("coefficient ring, warp B", t, ctag)
                    o4 = sb2.step(o3, cf4, p, dt, cubic_half)
                    r = t - lag_b
                    if hy <= r < hy + NY and ys + r - hy < Ly:
                        y = ys + r - hy
                        for cc in np.nonzero(col_ok)[0]:
                            assert np.isnan(out[y, x0 + cc]), ("written twice", y, x0 + cc)
                            out[y, x0 + cc] = o4[cc]
                # barrier after every second tick: the hand-over becomes visible
                if t % 2 == 1:
                    for (kind, slot), val in writes.items():
                        hand[slot] = val
                    writes = {}
    return out


def oracle_fd(p, phi, u, nsub):
    dt = 1.0 / p.m
    for _ in range(nsub):
        phi = O.diffuse(p, O.advect(p, phi, u, dt), phi, dt)
    return phi


@pytest.mark.parametrize("shape,NY", [((40, 128), 16), ((37, 212), 11), ((20, 64), 32),
                                      ((9, 96), 4), ((64, 300), 25)])
@pytest.mark.parametrize("sub", [2, 4])
def test_wave_model_equals_oracle_substeps(shape, NY, sub):
    Ly, Lx = shape
    rng = np.random.default_rng(Ly * 1000 + Lx + sub)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((2,) + shape)
    u[:, ::3, ::5] = 0.0  # u = 0 takes the kernel's else branches
    p = O.Params(Lx=Lx, Ly=Ly, m=4)
    got = wave_model(phi, u, p, sub, NY)
    assert not np.any(np.isnan(got))
    np.testing.assert_allclose(got, oracle_fd(p, phi, u, sub), rtol=0, atol=1e-13)


def test_wave_model_cubic_at_half():
    shape = (30, 128)
    rng = np.random.default_rng(11)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((2,) + shape)
    p = O.Params(Lx=128, Ly=30, m=4, cubic_at_half=1)
    got = wave_model(phi, u, p, 4, 12, cubic_half=True)
    np.testing.assert_allclose(got, oracle_fd(p, phi, u, 4), rtol=0, atol=1e-13)


def test_wave_model_detects_a_wrong_lag():
    """A planted mistake in the model's schedule (warp B's output row one tick
    early or late) must fail the comparison: the lag arithmetic is what this
    checks."""
    shape = (24, 128)
    rng = np.random.default_rng(3)
    phi = np.tanh(rng.standard_normal(shape))
    u = 0.05 * rng.standard_normal((2,) + shape)
    p = O.Params(Lx=128, Ly=24, m=4)
    ref = oracle_fd(p, phi, u, 4)
    for lag_b in (13, 15):
        with pytest.raises(AssertionError):
            got = wave_model(phi, u, p, 4, 12, lag_b=lag_b)
            assert not np.any(np.isnan(got))
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
