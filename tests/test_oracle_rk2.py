"""Pins of the RK2 step oracle (Sec. 2.1) composed of the pinned pieces (no GPU)."""
import dataclasses

import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I


@pytest.fixture(scope="module")
def rk2(oracle):
    from oracle import rk2 as R
    return R


def cfl_dt(prob, courant=0.2):
    h = min(prob.dx.min(), prob.dy.min(), prob.dz.min())
    return courant * h / max(np.abs(prob.u).max(), np.abs(prob.v).max(), np.abs(prob.w).max())


def test_step_ends_divergence_free(rk2, oracle):
    # Eqs. poisson2 and runge2: u^{k+1} has zero net flux in every merge group of the stage-2
    # operator (the divergence check does not involve rho)
    p = I.tiny_sphere(n=8)
    p.dt = cfl_dt(p)
    phi, (u, v, w), P2, (P1, ust, phis), s2 = rk2.rk2_step(p)
    p2 = dataclasses.replace(p, F=phis)
    div = oracle.divergence(p2, s2, u, v, w)
    scale = np.abs(s2.fold((s2.apertures[0] * np.abs(p.u))[:, :, 1:])).max() * p.dx.max() ** 2
    assert np.abs(div).max() <= 1e-12 * scale
    assert np.abs(oracle.divergence(p2, s2, p.u, p.v, p.w)).max() > 1e-3 * scale
    assert np.abs(phi - p.F).max() > 1e-4


def test_solenoidal_field_is_a_fixed_point_of_the_velocity_update(rk2, oracle):
    # with R = 0 and a field that is already projected, both pressures vanish and u^{k+1} = u^k;
    # phi^{k+1} is then one VOF step with u^k (the midpoint velocity is u^k)
    from oracle import vof
    p = I.tiny_sphere(n=8)
    p.dt = cfl_dt(p)
    s = oracle.System(p)
    u0, v0, w0 = oracle.project(p, s, s.solve_dense())
    q = dataclasses.replace(p, u=u0, v=v0, w=w0)
    q.dt = cfl_dt(q)
    phi, (u, v, w), P2, (P1, ust, phis), s2 = rk2.rk2_step(q)
    scale = np.abs(u0).max()
    assert np.abs(P1).max() <= 1e-9 * np.abs(s.solve_dense()).max()
    for a, b in ((u, u0), (v, v0), (w, w0)):
        assert np.abs(a - b).max() <= 1e-9 * scale
    ref = vof.advect(q, dt=q.dt)
    assert np.abs(phi - ref).max() <= 1e-9
