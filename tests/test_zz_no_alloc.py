"""vofp_residual_noalloc: the residual norm without device allocation.

Some callers cannot allocate device memory once set-up is over (their memory belongs to another
allocator's pool, or a fixed budget, or they cannot take cudaMalloc's device synchronisation).
For them the library offers vofp_residual_noalloc, whose only scratch is a fixed static device
array.  These tests call it through the C ABI on a freshly built context, check that calls after
the first leave device memory unchanged (the context's count, the driver's free bytes and the torch
allocator's reserve), and compare it with vofp_residual, which computes the same norm with
allocated scratch, on two calls in a row.  This file is collected last so that
a run stopping at its first failure has already run every other test.
"""
import gc

import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vofp():
    import __graft_entry__ as g
    g.build()
    from paper_1410_1937_gb300 import vofp as V
    return V


def _problem():
    # slender hull in waves: merge groups, cells without an unknown, ragged tiles
    return I.config2(shape=(96, 48, 40))


def _memory(ctx):
    """Device memory as three observers see it: the context's own count, the CUDA driver's free
    bytes, and the torch caching allocator's reserved bytes."""
    torch.cuda.synchronize()
    return (ctx.vofp_get_stats()["device_bytes"], torch.cuda.mem_get_info()[0],
            torch.cuda.memory_reserved())


def test_noalloc_residual_allocates_nothing_and_matches(vofp):
    prob = _problem()
    ctx, t = vofp.context_for(prob)
    assert ctx.vofp_get_stats()["groups"] > 0
    b = ctx.vofp_rhs_from_face_velocity(t["u"], t["v"], t["w"])
    x = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, prob.n)).cuda()
    gc.collect()
    gc.disable()   # no context of another test may be freed inside the measured span
    try:
        # first call on a freshly built context, before any solve or allocating residual: it may
        # load this entry point's code and static array onto the device (a one-time reservation
        # by the CUDA runtime); every later call must leave device memory exactly as it was
        first = ctx.vofp_residual_noalloc(b, x)
        before = _memory(ctx)
        second = ctx.vofp_residual_noalloc(b, x)
        third = ctx.vofp_residual_noalloc(b, x)
        after = _memory(ctx)
    finally:
        gc.enable()
    assert before == after, (before, after)
    assert first == second == third
    # the allocating entry point, called only now, gives the same norm
    ref = ctx.vofp_residual(b, x)
    assert ctx.vofp_get_stats()["device_bytes"] >= before[0]
    assert abs(first - ref) <= 1e-12 * ref
    # a solved pressure: a small residual, compared to the rounding of b - A x
    xs, info = ctx.vofp_solve(b, rtol=1e-10)
    ref_s = ctx.vofp_residual(b, xs)
    got_a = ctx.vofp_residual_noalloc(b, xs)
    got_b = ctx.vofp_residual_noalloc(b, xs)
    assert got_a == got_b
    assert abs(got_a - ref_s) <= 1e-13 + 1e-3 * ref_s
    assert got_a <= 1e-10


def test_noalloc_residual_rejects_too_many_merge_groups(vofp):
    # every fourth cell along x is small and merges into its -x neighbour: 69632 groups
    nx, ny, nz = 128, 128, 17
    prob = I.manufactured(2)
    prob.dx, prob.dy, prob.dz = np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny), np.full(nz, 1.0 / nz)
    prob.F = np.ones((nz, ny, nx))
    prob.vf = np.ones((nz, ny, nx))
    prob.vf[:, :, 1::4] = 0.05
    prob.ax, prob.ay, prob.az = np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)), np.ones((nz + 1, ny, nx))
    prob.u, prob.v, prob.w = np.zeros_like(prob.ax), np.zeros_like(prob.ay), np.zeros_like(prob.az)
    prob.merge_threshold = 0.1
    ctx, t = vofp.context_for(prob)
    assert ctx.vofp_get_stats()["groups"] == nz * ny * nx // 4
    b = torch.ones(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(vofp.VofpError) as e:
        ctx.vofp_residual_noalloc(b, b)
    assert e.value.status == vofp.ERR_INVALID_ARG
    assert "merge groups" in str(e.value)
