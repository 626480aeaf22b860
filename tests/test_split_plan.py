"""Work split of the colour-compact red-black iteration kernel (host logic, no GPU): the plan from
vofp_rbc_split_plan is walked with the kernel's own loop-header arithmetic, block by block, and
every (tile, plane) must be marched exactly once by at most `slots` blocks; the blocks of a group
march the same planes in the same steps."""
import pytest

SEG_STEPS = 6   # plane steps a column segment costs besides its planes (prologue + two closing t)


@pytest.fixture(scope="module")
def vofp():
    from paper_1410_1937_gb300 import build as B
    B.build()
    from paper_1410_1937_gb300 import vofp as V
    return V


def walk(tx, ty, nz, blocks, per, pad, gx=1, gy=1):
    """Segments ((tile x, tile y), k0, k1) of every block, as the kernel's loop header forms them."""
    nzp = nz + pad
    gsz = gx * gy
    ncx = tx // gx
    ncols = ncx * (ty // gy)
    total = ncols * nzp
    out = []
    for b in range(blocks):
        grp, jg = divmod(b, gsz)
        w0 = min(grp * per, total)
        w1 = min(w0 + per, total)
        w, segs = w0, []
        while w < w1:
            col = w // nzp
            kp0 = w - col * nzp
            kp1 = min(nzp, kp0 + (w1 - w))
            w += kp1 - kp0
            k0, k1 = max(kp0 - pad, 0), kp1 - pad
            if k1 > k0:
                tile = ((col % ncx) * gx + jg % gx, (col // ncx) * gy + jg // gx)
                segs.append((tile, k0, k1))
        out.append(segs)
    return out


def steps(segs):
    return sum(k1 - k0 + SEG_STEPS for _, k0, k1 in segs)


@pytest.mark.parametrize("tx,ty,nz,slots", [
    (8, 16, 128, 304),    # 512 x 256 x 128, 32 x 16 tiles, on 152 SMs x 2 blocks
    (8, 32, 128, 608), (16, 16, 256, 304), (6, 10, 50, 300),
    (8, 32, 100, 608), (8, 32, 200, 608), (16, 64, 256, 608),
    (2, 8, 64, 608), (2, 6, 40, 608), (4, 16, 64, 608), (1, 1, 1, 1), (3, 5, 7, 2), (1, 9, 300, 456),
    (5, 1, 33, 152), (7, 3, 1, 608),
])
def test_plan_marches_every_plane_once(vofp, tx, ty, nz, slots):
    blocks, per, pad, gx, gy = vofp.vofp_rbc_split_plan(tx, ty, nz, slots)
    assert 1 <= blocks <= slots and per >= 1 and 0 <= pad <= 2 * SEG_STEPS
    assert tx % gx == 0 and ty % gy == 0 and blocks % (gx * gy) == 0
    ncols = (tx // gx) * (ty // gy)
    groups = blocks // (gx * gy)
    assert (groups - 1) * per < ncols * (nz + pad) <= groups * per
    seen = {}
    plans = walk(tx, ty, nz, blocks, per, pad, gx, gy)
    for segs in plans:
        for tile, k0, k1 in segs:
            assert 0 <= tile[0] < tx and 0 <= tile[1] < ty
            for k in range(k0, k1):
                seen[tile, k] = seen.get((tile, k), 0) + 1
    assert len(seen) == tx * ty * nz and all(v == 1 for v in seen.values())
    # the members of a group march the same planes in the same order
    for g in range(groups):
        members = plans[g * gx * gy:(g + 1) * gx * gy]
        assert all([(k0, k1) for _, k0, k1 in m] == [(k0, k1) for _, k0, k1 in members[0]] for m in members)


def group_worst(tx, ty, nz, blocks, per, pad, gx, gy):
    return max(steps(s) for s in walk(tx, ty, nz, blocks, per, pad, gx, gy))


def equal_split_worst(tx, ty, nz, slots):
    total = tx * ty * nz
    n = max(1, min(slots, total))
    per = -(-total // n)
    return group_worst(tx, ty, nz, -(-total // per), per, 0, 1, 1)


def misaligned_edges(tx, ty, nz, per, pad, gx, gy):
    """(x edges, y edges) between tiles marched more than three steps apart."""
    nzp, ncx, ncy = nz + pad, tx // gx, ty // gy

    def apart(dist):
        r = dist % per
        return min(r, per - r) > 3
    ex = (ncx - 1) * ty if apart(nzp) else 0
    ey = (ncy - 1) * tx if apart(ncx * nzp) else 0
    return ex, ey


def test_full_size_plan_keeps_neighbours_in_step(vofp):
    """512 x 256 x 128 with 32 x 16 tiles (8 x 16 tiles, 128 planes, 304 resident blocks): the
    longest block marches 63 plane steps against 66 for equal planes per block, and the groups
    leave at most a quarter of the tile edges with their two sides marched apart (one tile per
    block leaves every x edge apart: the next tile column is nz + pad items on, 21 steps off a
    multiple of per)."""
    blocks, per, pad, gx, gy = vofp.vofp_rbc_split_plan(8, 16, 128, 304)
    assert group_worst(8, 16, 128, blocks, per, pad, gx, gy) == 63
    assert equal_split_worst(8, 16, 128, 304) == 66
    ex, ey = misaligned_edges(8, 16, 128, per, pad, gx, gy)
    edges = 7 * 16 + 15 * 8
    assert (ex + ey) <= edges / 4
    ex1, ey1 = misaligned_edges(8, 16, 128, 56, 5, 1, 1)
    assert ex1 == 7 * 16


@pytest.mark.parametrize("nz", [100, 200])
def test_plan_keeps_more_edges_in_step_than_the_equal_split(vofp, nz):
    """For 100 or 200 planes the equal split puts every neighbour pair of tiles apart; the plan
    keeps most of them in step at no more plane steps."""
    tx, ty = 8, 16
    eq_per = -(-tx * ty * nz // 304)
    assert sum(misaligned_edges(tx, ty, nz, eq_per, 0, 1, 1)) == 7 * 16 + 15 * 8
    blocks, per, pad, gx, gy = vofp.vofp_rbc_split_plan(tx, ty, nz, 304)
    assert sum(misaligned_edges(tx, ty, nz, per, pad, gx, gy)) <= (7 * 16 + 15 * 8) / 3
    assert group_worst(tx, ty, nz, blocks, per, pad, gx, gy) <= equal_split_worst(tx, ty, nz, 304)


def test_plan_rejects_bad_arguments(vofp):
    L = vofp._lib
    import ctypes
    v = [ctypes.c_int() for _ in range(5)]
    r = [ctypes.byref(x) for x in v]
    assert L.vofp_rbc_split_plan(8, 32, 128, 608, *r) == vofp.OK
    assert L.vofp_rbc_split_plan(0, 32, 128, 608, *r) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(8, 32, 128, 0, *r) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(8, 32, 128, 608, None, *r[1:]) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(8, 32, 128, 608, *r[:4], None) == vofp.ERR_INVALID_ARG
    assert L.vofp_rbc_split_plan(1 << 20, 1 << 10, 128, 608, *r) == vofp.ERR_INVALID_ARG
