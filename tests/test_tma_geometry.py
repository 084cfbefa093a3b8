"""The TMA collide kernel's tile geometry (csrc/collide2d_tma.cu), restated
and checked on the CPU against the pull-streaming definition
f_i(r, t) = buf_i(r - e_i) and the copy engine's rules: for FP32 and FP16
storage, every plane's box starts on a 16-byte boundary in x, the column a
thread reads holds the population pulled from x - e_x, the boxes tile the
shared memory back to back with 128-byte-aligned starts, and the expected
transaction bytes are the boxes' sum."""
import pytest

# D2Q9 order of the library: 0 rest; 1..4 (1,0),(0,1),(-1,0),(0,-1); 5..8 (1,1),(-1,1),(-1,-1),(1,-1)
E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
TT = 32
PHW, PHH = 40, 36


def geometry(elem):
    A = 16 // elem
    w = [TT if ex == 0 else TT + A for ex, _ in E]
    dx = [-A if ex > 0 else 0 for ex, _ in E]
    col = [A - 1 if ex > 0 else (1 if ex < 0 else 0) for ex, _ in E]
    nshift = [sum(1 for j in range(i) if E[j][0] != 0) for i in range(10)]
    off = [TT * (TT * i + A * nshift[i]) for i in range(10)]  # elements
    return w, dx, col, off


@pytest.mark.parametrize("elem", [4, 2])
def test_boxes_hold_the_pulled_populations(elem):
    w, dx, col, off = geometry(elem)
    for x0 in range(0, 4 * TT, TT):
        for i, (ex, ey) in enumerate(E):
            assert ((x0 + dx[i]) * elem) % 16 == 0, (elem, i)  # copy origin on 16 bytes
            assert (w[i] * elem) % 16 == 0  # inner box extent
            for tx in range(TT):
                c = tx + col[i]
                assert 0 <= c < w[i]
                assert x0 + dx[i] + c == (x0 + tx) - ex  # the column holds buf_i(x - e_x)
            # rows: the box starts at y0 - e_y, so row ly holds buf_i(y0 + ly - e_y)


@pytest.mark.parametrize("elem", [4, 2])
def test_planes_tile_shared_memory(elem):
    w, dx, col, off = geometry(elem)
    for i in range(9):
        assert off[i + 1] - off[i] == TT * w[i]  # plane i's box is TT rows of w[i]
        assert (off[i] * elem) % 128 == 0  # copy destinations 128-byte aligned
    pop_bytes = off[9] * elem
    assert pop_bytes == sum(TT * wi * elem for wi in w)
    assert (128 + pop_bytes) % 128 == 0  # the phi box follows, aligned too
    tx_bytes = pop_bytes + 4 * PHW * PHH
    assert tx_bytes == sum(TT * wi * elem for wi in w) + 4 * PHW * PHH


def test_phi_box_covers_the_halo():
    # phi box: columns x0 - 4 .. x0 + 35, rows y0 - 2 .. y0 + 33; mu on the tile + 1
    # needs phi on the tile + 2: columns x0 - 2 .. x0 + 33
    assert ((0 - 4) * 4) % 16 == 0
    lo, hi = -4, -4 + PHW - 1
    assert lo <= -2 and hi >= TT + 1
    assert -2 + PHH - 1 == TT + 1


# ---- the edge fixups of the TMA collide kernels -----------------------------------------
# (the pipelined kernels' 32 x 16 tiles, loaded into at most 3 + 2 register slots per
# thread before the copy wait; the one-tile kernels' 32 x 32 tiles, after it)


def phi_fix_cells(Lx, Ly, x0, y0, PY=16):
    """The phi box cells (rx, ry) of tile (x0, y0) that the edge fixup loads,
    in its order: the column strips (all PY + 4 rows), then the row strips
    between them."""
    PPHH = PY + 4
    rxr, ryb = Lx - x0 + 2, Ly - y0 + 2
    wl, wr = (2 if x0 == 0 else 0), max(0, TT + 4 - rxr)
    ht, hb = (2 if y0 == 0 else 0), max(0, PPHH - ryb)
    if wl + wr + ht + hb == 0:
        return []
    ncol, wc = PPHH * (wl + wr), TT + 4 - wl - wr
    ntot = ncol + (ht + hb) * wc
    if PY == 16:
        assert ntot <= 3 * 256  # three slots per thread
    out = []
    for q in range(ntot):
        if q < ncol:
            c, ry = divmod(q, PPHH)
            rx = c if c < wl else rxr + (c - wl)
        else:
            r, cx = divmod(q - ncol, wc)
            rx, ry = wl + cx, (r if r < ht else ryb + (r - ht))
        out.append((rx, ry))
    return out


def pop_fix_cells(Lx, Ly, x0, y0, PY=16):
    """(i, xs, ys) of the populations pulled across the lattice's edges that
    the edge fixup loads (8 planes x (PY + TT) candidates, two slots)."""
    out = []
    for q in range(8 * (PY + TT)):
        assert q < 2 * 256
        i, j = 1 + q // (PY + TT), q % (PY + TT)
        ex, ey = E[i]
        if j < PY:
            if ex == 0:
                continue
            xs, ys = (0 if ex > 0 else Lx - 1), y0 + j
        else:
            if ey == 0:
                continue
            ys, xs = (0 if ey > 0 else Ly - 1), x0 + j - PY
        if xs < x0 or xs >= x0 + TT or xs >= Lx or ys < y0 or ys >= y0 + PY or ys >= Ly:
            continue
        out.append((i, xs, ys))
    return out


@pytest.mark.parametrize("PY", [16, 32])
@pytest.mark.parametrize("Lx,Ly", [(64, 64), (68, 80), (100, 64), (128, 132), (96, 200), (260, 68)])
def test_edge_fixups_cover_exactly_the_cells_the_copies_zero(Lx, Ly, PY):
    """Every phi cell of a tile's 36 x 20 box outside the lattice is loaded
    exactly once (and no inside cell), its periodic image within one
    conditional wrap; every population of the tile whose pull buf_i(r - e_i)
    crosses an edge is loaded, and no other."""
    PPHH = PY + 4
    for y0 in range(0, Ly, PY):
        for x0 in range(0, Lx, TT):
            cells = phi_fix_cells(Lx, Ly, x0, y0, PY)
            assert len(cells) == len(set(cells))
            outside = {(rx, ry) for ry in range(PPHH) for rx in range(TT + 4)
                       if not (0 <= x0 - 2 + rx < Lx and 0 <= y0 - 2 + ry < Ly)}
            assert set(cells) == outside, (x0, y0)
            for rx, ry in cells:
                gx, gy = x0 - 2 + rx, y0 - 2 + ry
                assert -Lx <= gx < 2 * Lx and -Ly <= gy < 2 * Ly  # wrap1's range
                assert PHW * ry + rx + 2 < PHW * PPHH
            crossing = set()
            for ys in range(y0, min(y0 + PY, Ly)):
                for xs in range(x0, min(x0 + TT, Lx)):
                    for i in range(1, 9):
                        sx, sy = xs - E[i][0], ys - E[i][1]
                        if not (0 <= sx < Lx and 0 <= sy < Ly):
                            crossing.add((i, xs, ys))
            assert set(pop_fix_cells(Lx, Ly, x0, y0, PY)) == crossing, (x0, y0)
