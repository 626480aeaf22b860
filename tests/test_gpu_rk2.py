"""GPU parity of one and two RK2 steps (Sec. 2.1) through vofp_rk2_step against oracle/rk2.py."""
import dataclasses

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_two_rk2_steps_match_oracle(vofp, oracle, mode):
    from oracle import rk2
    prob = I.tiny_sphere(n=16)
    h = prob.dx.min()
    prob.dt = 0.2 * h / max(np.abs(prob.u).max(), np.abs(prob.v).max(), np.abs(prob.w).max())
    # momentum terms keep every step's right-hand side away from zero (a projected field alone
    # gives the next step's first solve a right-hand side at rounding level)
    R = I.momentum_terms(prob)
    Rd = tuple(dev(a) for a in R)
    ctx, t = vofp.context_for(prob)
    p = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    kw = (dict(mode=vofp.MODE_FP64, rtol=1e-12, precond=vofp.PRECOND_JACOBI) if mode == "fp64"
          else dict(mode=vofp.MODE_MIXED, rtol=1e-10, precond=vofp.PRECOND_RBSGS))
    tol = 1e-8 if mode == "fp64" else 1e-6
    cur = prob
    for step in range(2):
        i1, i2, mx = ctx.vofp_rk2_step(t["F"], t["ax"], t["ay"], t["az"], t["vf"], t["u"], t["v"], t["w"], cur.bc, p,
                                       order=step % 2, R=Rd, rho_liquid=cur.rho_liquid, rho_gas=cur.rho_gas,
                                       merge_threshold=cur.merge_threshold, dt=cur.dt, **kw)
        assert i1["status"] == 0 and i2["status"] == 0
        phi, (u, v, w), P2, _, s2 = rk2.rk2_step(cur, order=step % 2, R=R)
        pg = p.cpu().numpy().reshape(prob.shape)
        assert np.linalg.norm(pg - P2) <= tol * np.linalg.norm(P2)
        for got, ref in ((t["u"], u), (t["v"], v), (t["w"], w)):
            g = got.cpu().numpy().reshape(ref.shape)
            assert np.abs(g - ref).max() <= tol * np.abs(ref).max()
        assert np.abs(t["F"].cpu().numpy().reshape(prob.shape) - phi).max() <= tol
        cur = dataclasses.replace(cur, F=phi, u=u, v=v, w=w)
    # the second step started from the first step's pressure
    assert i1["iterations"] > 0
    ctx.close()
