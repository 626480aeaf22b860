"""Full-size parity on the 512x256x128 hull-in-waves workload, in the configuration bench.py times.

The oracle assembles this system on the host (about 16.8 M cells) but a full oracle solve would
take minutes, so the solutions are checked through properties that hold at any size: the oracle's
own residual ||b_hat - A_hat x|| / ||b_hat|| of the GPU pressure.  The right-hand side, the merge
map and one operator apply are compared element by element.
"""
import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup(oracle):
    import __graft_entry__ as g
    g.build()
    from paper_1410_1937_gb300 import vofp
    prob = I.config2()
    sysm = oracle.System(prob)
    ctx, t = vofp.context_for(prob)
    b = ctx.vofp_rhs_from_face_velocity(t["u"], t["v"], t["w"])
    return vofp, prob, sysm, ctx, b


def test_fullsize_rhs_and_merge_map(setup):
    vofp, prob, s, ctx, b = setup
    bg = b.cpu().numpy()
    assert np.abs(bg - s.b).max() <= 1e-13 * np.abs(s.b).max()
    np.testing.assert_array_equal(ctx.vofp_merge_map().cpu().numpy(), s.root.astype(np.int32))


def test_fullsize_apply(setup):
    vofp, prob, s, ctx, b = setup
    x = np.random.default_rng(21).uniform(-1, 1, prob.n)
    y = ctx.vofp_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = s.apply_full(x).ravel()
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("mode,precond,rtol", [("mixed", "rbsgs", 1e-8), ("fp64", "jacobi", 1e-10),
                                               ("fp64", "rbsgs", 1e-10), ("mixed", "jacobi", 1e-8)])
def test_fullsize_solution_residual_by_oracle(setup, mode, precond, rtol):
    vofp, prob, s, ctx, b = setup
    m = vofp.MODE_MIXED if mode == "mixed" else vofp.MODE_FP64
    pc = vofp.PRECOND_RBSGS if precond == "rbsgs" else vofp.PRECOND_JACOBI
    x, info = ctx.vofp_solve(b, rtol=rtol, mode=m, precond=pc)
    assert info["status"] == 0, info
    res = s.residual(x.cpu().numpy())
    assert res <= rtol * 1.01, (res, info)
    assert abs(res - info["rel_residual"]) <= 1e-3 * res + 1e-16


def test_fullsize_projection(setup, oracle):
    """Projection of the face velocities with the mixed-precision pressure (Sec. 2.1 Eq. runge1),
    face by face against the oracle on the same pressure; the projected field's group divergence
    is the pressure equation's residual times dt (rtol 1e-8 of b_hat)."""
    vofp, prob, s, ctx, b = setup
    u, v, w = (torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda() for a in (prob.u, prob.v, prob.w))
    x, info = ctx.vofp_solve(b, rtol=1e-8, mode=vofp.MODE_MIXED)
    assert info["status"] == 0
    uo, vo, wo, div, mx = ctx.vofp_project(x, u, v, w)
    ru, rv, rw = oracle.project(prob, s, x.cpu().numpy().reshape(prob.shape))
    for got, ref in ((uo, ru), (vo, rv), (wo, rw)):
        g = got.cpu().numpy().reshape(ref.shape)
        assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()
    # sum over groups of div^2 = dt^2 ||b_hat - A_hat x||^2 (the residual identity of the projection)
    gdiv = div.cpu().numpy()
    assert abs(np.linalg.norm(gdiv) - prob.dt * np.linalg.norm(s.bhat) * info["rel_residual"]) <= \
        1e-3 * prob.dt * np.linalg.norm(s.bhat) * info["rel_residual"]
