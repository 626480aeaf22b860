"""Work split of the colour-compact red-black iteration kernel (host logic, no GPU): the plan from
vofp_rbc_split_plan is walked with the kernel's own loop-header arithmetic, block by block, and
every (tile, plane) must be marched exactly once by at most `slots` blocks."""
import pytest

SEG_STEPS = 5   # plane steps a tile-column segment costs besides its planes (prologue + closing t)


@pytest.fixture(scope="module")
def vofp():
    from paper_1410_1937_gb300 import build as B
    B.build()
    from paper_1410_1937_gb300 import vofp as V
    return V


def walk(tiles, nz, blocks, per, pad):
    """Segments (tile, k0, k1) of every block, as the kernel's loop header forms them."""
    nzp = nz + pad
    total = tiles * nzp
    out = []
    for b in range(blocks):
        w0 = min(b * per, total)
        w1 = min(w0 + per, total)
        w, segs = w0, []
        while w < w1:
            t = w // nzp
            kp0 = w - t * nzp
            kp1 = min(nzp, kp0 + (w1 - w))
            w += kp1 - kp0
            k0, k1 = max(kp0 - pad, 0), kp1 - pad
            if k1 > k0:
                segs.append((t, k0, k1))
        out.append(segs)
    return out


def steps(segs):
    return sum(k1 - k0 + SEG_STEPS for _, k0, k1 in segs)


@pytest.mark.parametrize("tx,ty,nz,slots", [
    (8, 32, 128, 608),    # 512 x 256 x 128 on 152 SMs x 4 blocks
    (8, 32, 100, 608), (8, 32, 200, 608), (16, 64, 256, 608),
    (2, 8, 64, 608), (2, 6, 40, 608), (4, 16, 64, 608), (1, 1, 1, 1), (3, 5, 7, 2), (1, 9, 300, 456),
    (5, 1, 33, 152), (7, 3, 1, 608),
])
def test_plan_marches_every_plane_once(vofp, tx, ty, nz, slots):
    blocks, per, pad = vofp.vofp_rbc_split_plan(tx, ty, nz, slots)
    assert 1 <= blocks <= slots and per >= 1 and 0 <= pad <= 2 * SEG_STEPS
    tiles = tx * ty
    assert (blocks - 1) * per < tiles * (nz + pad) <= blocks * per
    seen = [[0] * nz for _ in range(tiles)]
    for segs in walk(tiles, nz, blocks, per, pad):
        for t, k0, k1 in segs:
            for k in range(k0, k1):
                seen[t][k] += 1
    assert all(v == 1 for row in seen for v in row)


def equal_split_worst(tiles, nz, slots):
    total = tiles * nz
    n = max(1, min(slots, total))
    per = -(-total // n)
    return max(steps(s) for s in walk(tiles, nz, -(-total // per), per, 0))


def test_full_size_plan_beats_the_equal_split_and_keeps_y_neighbours_in_step(vofp):
    """512 x 256 x 128 (8 x 32 tiles, 128 planes, 608 resident blocks): the longest block marches 61
    plane steps against 64 for equal planes per block, and a tile's y-neighbours (8 tile columns,
    8 (nz + pad) work items away) are a whole number of blocks away, so they are marched at the
    same plane in the same step."""
    blocks, per, pad = vofp.vofp_rbc_split_plan(8, 32, 128, 608)
    worst = max(steps(s) for s in walk(256, 128, blocks, per, pad))
    assert worst == 61 and equal_split_worst(256, 128, 608) == 64
    assert (8 * (128 + pad)) % per == 0


@pytest.mark.parametrize("nz", [100, 200])
def test_plan_keeps_y_neighbours_in_step_where_the_equal_split_does_not(vofp, nz):
    """For 100 or 200 planes the equal split puts y-neighbour tiles 12 or more steps apart (their halo
    rows then come from DRAM); the plan keeps them within three steps at no more plane steps."""
    tiles = 256
    eq_per = -(-tiles * nz // 608)
    d = (8 * nz) % eq_per
    assert min(d, eq_per - d) > 3
    blocks, per, pad = vofp.vofp_rbc_split_plan(8, 32, nz, 608)
    d = (8 * (nz + pad)) % per
    assert min(d, per - d) <= 3
    assert max(steps(s) for s in walk(tiles, nz, blocks, per, pad)) <= equal_split_worst(tiles, nz, 608)


def test_plan_rejects_bad_arguments(vofp):
    L = vofp._lib
    import ctypes
    b, p, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ok = L.vofp_rbc_split_plan(8, 32, 128, 608, ctypes.byref(b), ctypes.byref(p), ctypes.byref(q))
    assert ok == vofp.OK
    assert L.vofp_rbc_split_plan(0, 32, 128, 608, ctypes.byref(b), ctypes.byref(p), ctypes.byref(q)) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(8, 32, 128, 0, ctypes.byref(b), ctypes.byref(p), ctypes.byref(q)) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(8, 32, 128, 608, None, ctypes.byref(p), ctypes.byref(q)) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(1 << 20, 1 << 10, 128, 608, ctypes.byref(b), ctypes.byref(p),
                                 ctypes.byref(q)) == vofp.ERR_INVALID_ARG
