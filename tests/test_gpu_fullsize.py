"""Parity at the workloads' own sizes, in the configuration bench.py times.

The 128x64x64 stretched grid around a half-immersed sphere and the 512x256x128 slender hull in
waves are solved by every GPU variant and compared element by element with the oracle's solution
(plain FP64 Jacobi-PCG on the host cores to relative residual 1e-12): the gate is a relative L2
error of at most 1e-6, at residual 1e-10 for the FP64 solves and 1e-8 for the mixed-precision
ones, with the residual recomputed by the oracle.  The oracle solve of the large grid takes a
couple of minutes on the host cores; it runs once per module.  The right-hand side, the merge map,
one operator apply and the projection are compared element by element as well.  The
1024x512x256 case (134 M cells) is checked through the oracle's residual of the GPU pressure.
"""

import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GATE = 1e-6
VARIANTS = [("fp64", "jacobi", 1e-10), ("fp64", "rbsgs", 1e-10), ("mixed", "jacobi", 1e-8),
            ("mixed", "rbsgs", 1e-8)]


def _vofp():
    import __graft_entry__ as g
    g.build()
    from paper_1410_1937_gb300 import vofp
    return vofp


@pytest.fixture(scope="module", params=["c1-128x64x64", "c2-512x256x128"])
def case(request, oracle):
    vofp = _vofp()
    prob = I.config1() if request.param.startswith("c1") else I.config2()
    sysm = oracle.System(prob)
    oracle.set_threads(0)
    xref, info = sysm.solve_pcg(rtol=1e-12)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12, info
    ctx, t = vofp.context_for(prob)
    b = ctx.vofp_rhs_from_face_velocity(t["u"], t["v"], t["w"])
    yield vofp, prob, sysm, ctx, t, b, xref.ravel()
    ctx.close()


def test_rhs_and_merge_map(case):
    vofp, prob, s, ctx, t, b, xref = case
    bg = b.cpu().numpy()
    assert np.abs(bg - s.b).max() <= 1e-13 * np.abs(s.b).max()
    np.testing.assert_array_equal(ctx.vofp_merge_map().cpu().numpy(), s.root.astype(np.int32))


def test_apply(case):
    vofp, prob, s, ctx, t, b, xref = case
    x = np.random.default_rng(21).uniform(-1, 1, prob.n)
    y = ctx.vofp_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = s.apply_full(x).ravel()
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("mode,precond,rtol", VARIANTS)
def test_solution_error_against_oracle(case, mode, precond, rtol):
    """Relative L2 error of the GPU pressure against the oracle's 1e-12 solution, every cell."""
    vofp, prob, s, ctx, t, b, xref = case
    m = vofp.MODE_MIXED if mode == "mixed" else vofp.MODE_FP64
    pc = vofp.PRECOND_RBSGS if precond == "rbsgs" else vofp.PRECOND_JACOBI
    x, info = ctx.vofp_solve(b, rtol=rtol, mode=m, precond=pc)
    assert info["status"] == 0, info
    xg = x.cpu().numpy()
    res = s.residual(xg)
    assert res <= rtol, (res, info)
    assert abs(res - info["rel_residual"]) <= 1e-3 * res + 1e-16
    err = np.linalg.norm(xg - xref) / np.linalg.norm(xref)
    print(f"{prob.name} {mode}+{precond} rtol {rtol:g}: residual {res:.3e}, error {err:.3e}, "
          f"{info['iterations']} iterations")
    assert err <= GATE, (err, res, info)


def test_projection(case, oracle):
    """Projection of the face velocities with the mixed-precision pressure (Sec. 2.1 Eq. runge1),
    face by face against the oracle on the same pressure; the projected field's group divergence
    is the pressure equation's residual times dt."""
    vofp, prob, s, ctx, t, b, xref = case
    x, info = ctx.vofp_solve(b, rtol=1e-8, mode=vofp.MODE_MIXED)
    assert info["status"] == 0
    uo, vo, wo, div, mx = ctx.vofp_project(x, t["u"], t["v"], t["w"])
    ru, rv, rw = oracle.project(prob, s, x.cpu().numpy().reshape(prob.shape))
    for got, ref in ((uo, ru), (vo, rv), (wo, rw)):
        g = got.cpu().numpy().reshape(ref.shape)
        assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()
    # sum over groups of div^2 = dt^2 ||b_hat - A_hat x||^2 (the residual identity of the projection)
    gdiv = div.cpu().numpy()
    assert abs(np.linalg.norm(gdiv) - prob.dt * np.linalg.norm(s.bhat) * info["rel_residual"]) <= \
        1e-3 * prob.dt * np.linalg.norm(s.bhat) * info["rel_residual"]


def _host_memory_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def test_largest_case_residual_by_oracle(oracle):
    """1024x512x256 (134 M cells), mixed red-black to 1e-8: the oracle assembles the same system
    on the host and recomputes the residual of the GPU pressure (a solve by the oracle would take
    about half an hour on the host cores)."""
    if _host_memory_gb() < 160:
        pytest.skip("the oracle's assembly of 134 M cells needs about 100 GB of host memory")
    vofp = _vofp()
    prob = I.config4()
    ctx, t = vofp.context_for(prob)
    b = ctx.vofp_rhs_from_face_velocity(t["u"], t["v"], t["w"])
    x, info = ctx.vofp_solve(b, rtol=1e-8, mode=vofp.MODE_MIXED, precond=vofp.PRECOND_RBSGS)
    assert info["status"] == 0, info
    xg = x.cpu().numpy()
    ctx.close()
    del t, b, x
    torch.cuda.empty_cache()
    s = oracle.System(prob)
    res = s.residual(xg)
    print(f"{prob.name}: residual by the oracle {res:.3e}, GPU {info['rel_residual']:.3e}, "
          f"{info['iterations']} iterations, {info['seconds']:.2f} s")
    assert res <= 1e-8
    assert abs(res - info["rel_residual"]) <= 1e-3 * res
