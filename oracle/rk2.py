"""Oracle: one second-order Runge-Kutta step of Sec. 2.1 around the pressure solve, composed of
the oracle's own pieces (poisson.System / solve_dense / project and vof.advect), FP64, CPU.

TEST INFRASTRUCTURE ONLY (imported by tests/ alone).

Stage 1: operator with rho(phi^k); P* for the face field u^k + dt R (Eq. poisson1); u* = that
field - dt grad P* / rho (Eq. runge1); phi* = phi^k - VOF(u^k, phi^k, dt).
Stage 2: operator with rho(phi*); P^{k+1} for the face field u* + u^k + dt R (Eq. poisson2);
u^{k+1} = (that field - dt grad P^{k+1} / rho) / 2 (Eq. runge2); phi^{k+1} = phi^k -
VOF((u* + u^k) / 2, phi^k, dt).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import poisson, vof


def rk2_step(prob, order=0, R=None):
    """Returns (phi^{k+1}, (u, v, w)^{k+1}, P^{k+1}, stage-1 results (P*, u*, phi*), the stage-2
    system)."""
    dt = prob.dt
    vel = (np.asarray(prob.u, dtype=np.float64), np.asarray(prob.v, dtype=np.float64),
           np.asarray(prob.w, dtype=np.float64))
    Rs = (0.0, 0.0, 0.0) if R is None else R
    f1 = tuple(vel[a] + dt * Rs[a] for a in range(3))
    p1 = dataclasses.replace(prob, u=f1[0], v=f1[1], w=f1[2])
    s1 = poisson.System(p1)
    P1 = s1.solve_dense()
    ust = poisson.project(p1, s1, P1)
    phis = vof.advect(prob, dt=dt, order=order)
    f2 = tuple(ust[a] + vel[a] + dt * Rs[a] for a in range(3))
    p2 = dataclasses.replace(prob, F=phis, u=f2[0], v=f2[1], w=f2[2])
    s2 = poisson.System(p2)
    P2 = s2.solve_dense()
    uf = poisson.project(p2, s2, P2)
    unew = tuple(0.5 * uf[a] for a in range(3))
    mid = tuple(0.5 * (ust[a] + vel[a]) for a in range(3))
    phinew = vof.advect(prob, dt=dt, order=order, u=mid[0], v=mid[1], w=mid[2])
    return phinew, unew, P2, (P1, ust, phis), s2
