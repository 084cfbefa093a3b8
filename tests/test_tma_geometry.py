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
