"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test would fail under a plausible mistake in the oracle: a wrong face average (layered closed
form, manufactured solution), a wrong metric or half-cell Dirichlet distance (manufactured
solution, 1-D reduction), a sign or area error in the divergence (linear-velocity closed form,
projection), a wrong merge (triple product by brute force, handmade merge cases), or a wrong
solver (dense LU, Lanczos bounds).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1410_1937_gb300 import inputs as I


def cell_volumes(p):
    return p.dz[:, None, None] * p.dy[None, :, None] * p.dx[None, None, :]


def test_dense_lu_equals_pcg_on_tiny_sphere(oracle):
    p = I.tiny_sphere()
    s = oracle.System(p)
    assert s.M < p.n and (s.root < 0).any(), "the case must have merged and inactive cells"
    dense = s.solve_dense()
    pcg, info = s.solve_pcg(rtol=1e-13)
    assert info["status"] == 0
    assert np.linalg.norm(pcg - dense) <= 1e-12 * np.linalg.norm(dense)
    assert s.residual(dense) < 1e-14


def test_operator_symmetric_positive_definite(oracle):
    s = oracle.System(I.tiny_sphere())
    A = s.Ahat
    assert abs(A - A.T).max() == 0.0
    np.linalg.cholesky(A.toarray())
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(s.M), rng.standard_normal(s.M)
    assert abs(x @ (A @ y) - y @ (A @ x)) <= 1e-13 * abs(x @ (A @ y))


def test_merged_operator_is_group_sum_brute_force(oracle):
    # A_hat[I, J] = sum over cells i of group I and j of group J of A[i, j] (Sec. 2.3 merging)
    p = I.tiny_sphere(n=6, radius=0.27)
    s = oracle.System(p)
    A = s.A.toarray()
    groups = {}
    for c, r in enumerate(s.root):
        if r >= 0:
            groups.setdefault(int(r), []).append(c)
    assert any(len(g) > 1 for g in groups.values())
    masters = list(s.masters)
    Ah = s.Ahat.toarray()
    for a, I_ in enumerate(masters):
        for b, J_ in enumerate(masters):
            ref = 0.0
            for i in groups[int(I_)]:
                for j in groups[int(J_)]:
                    ref += A[i, j]
            assert abs(Ah[a, b] - ref) <= 1e-15 * max(1.0, abs(ref))
    b_full = s.b
    for a, I_ in enumerate(masters):
        assert abs(s.bhat[a] - sum(b_full[c] for c in groups[int(I_)])) < 1e-18 + 1e-14 * abs(s.bhat[a])


def _cond(A):
    ev = np.linalg.eigvalsh(A)
    return ev[-1] / ev[0]


def test_merging_improves_conditioning(oracle):
    # Sec. 2.3: merging cells of small cut volume improves the conditioning of the Poisson matrix
    p = I.tiny_sphere(n=8, threshold=0.25)
    merged = oracle.System(p).Ahat.toarray()
    p.merge_threshold = 0.0
    plain = oracle.System(p).Ahat.toarray()
    assert merged.shape[0] < plain.shape[0]
    assert _cond(merged) < _cond(plain)


def test_density_smoothing_improves_conditioning(oracle):
    # Sec. 2.10: smoothing rho with (1/4, 1/2, 1/4) along each axis improves the conditioning
    p = I.tiny_sphere(n=8, threshold=0.25)
    sharp = oracle.System(p).Ahat.toarray()
    p.density_smoothing = 1
    smooth = oracle.System(p).Ahat.toarray()
    d1, d2 = np.diag(sharp) ** -0.5, np.diag(smooth) ** -0.5
    assert _cond(smooth) < _cond(sharp)
    assert _cond(d2[:, None] * smooth * d2) < _cond(d1[:, None] * sharp * d1)


def test_smoothing_filter_conserves_interior_mass(oracle):
    F = np.zeros((5, 6, 7))
    F[2, 3, 3] = 1.0
    rho = oracle.density(F, 1.0, 0.0, smoothing=True)
    assert abs(rho.sum() - 1.0) < 1e-15 and abs(rho[2, 3, 3] - 0.125) < 1e-15


def test_smoothing_filter_reflects_at_the_wall(oracle):
    # Sec. 2.10's (1/4, 1/2, 1/4) filter at a domain wall takes the cell itself as the missing
    # neighbour (reading 4): an impulse in a corner cell keeps 3/4 per axis and passes 1/4 to its
    # one neighbour per axis, so the corner ends at (3/4)^3 and the mass is conserved.  Dropping
    # the missing neighbour (a zero there) would leave 1/2 per axis and lose mass.
    F = np.zeros((4, 5, 6))
    F[0, 0, 0] = 1.0
    rho = oracle.density(F, 3.0, 1.0, smoothing=True)   # rho = 1 + 2 * smoothed(F)
    w = np.array([0.75, 0.25])
    ref = np.ones_like(F)
    ref[:2, :2, :2] += 2.0 * w[:, None, None] * w[None, :, None] * w[None, None, :]
    np.testing.assert_allclose(rho, ref, rtol=0, atol=1e-15)
    # the far corner: same closed form mirrored
    F2 = F[::-1, ::-1, ::-1].copy()
    np.testing.assert_allclose(oracle.density(F2, 3.0, 1.0, smoothing=True), ref[::-1, ::-1, ::-1], atol=1e-15)


def test_manufactured_solution_second_order(oracle):
    errs = []
    for n in (8, 16, 32, 64):
        p = I.manufactured(n)
        s = oracle.System(p)
        b_full = I.manufactured_rhs(p).ravel()
        s.bhat = s.P.T @ b_full
        ph, info = s.solve_pcg(rtol=1e-13)
        exact = I.manufactured_pressure(p)
        errs.append(np.abs(ph - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.85 < r < 2.15 for r in rates), (errs, rates)


def test_layered_density_closed_form_with_stretched_cells(oracle):
    # Constant outward flux through layers of piecewise-constant density: the continuous solution
    # p(x) = g * integral_x^L rho ds is reproduced exactly by the half-cell harmonic face average;
    # an arithmetic mean of 1/rho would not.
    nx, ny, nz = 12, 3, 2
    xn = I.tanh_nodes(0.0, 1.0, nx, 0.3, 0.1)
    dx = np.diff(xn)
    rng = np.random.default_rng(5)
    Fx = rng.uniform(0, 1, nx)
    p = I.manufactured(2)
    p.dx, p.dy, p.dz = dx, np.array([0.2, 0.5, 0.3]), np.array([0.7, 0.4])
    p.F = np.broadcast_to(Fx[None, None, :], (nz, ny, nx)).copy()
    p.vf = np.ones((nz, ny, nx))
    p.ax, p.ay, p.az = np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)), np.ones((nz + 1, ny, nx))
    p.u, p.v, p.w = np.zeros_like(p.ax), np.zeros_like(p.ay), np.zeros_like(p.az)
    p.rho_liquid, p.rho_gas = 1000.0, 1.2
    g = 0.37
    s = oracle.System(p, neumann_flux=[np.full((nz, ny), g), None, None, None, None, None])
    ph = s.solve_dense()
    rho = 1.2 + (1000.0 - 1.2) * Fx
    exact = np.array([g * (rho[i] * dx[i] / 2 + (rho[i + 1:] * dx[i + 1:]).sum()) for i in range(nx)])
    np.testing.assert_allclose(ph, np.broadcast_to(exact, (nz, ny, nx)), rtol=1e-12)


def test_three_d_reduces_to_thomas_tridiagonal(oracle):
    # Everything varies in x only: every (j, k) line solves the same tridiagonal system.
    nx, ny, nz = 16, 4, 3
    xn = I.tanh_nodes(-1.0, 1.0, nx, 0.0, 0.2)
    dx = np.diff(xn)
    rng = np.random.default_rng(11)
    Fx = np.clip(rng.uniform(-0.5, 1.5, nx), 0, 1)
    ap = rng.uniform(0.2, 1.0, nx + 1)
    ux = rng.uniform(-1, 1, nx + 1)
    p = I.manufactured(2)
    p.dx, p.dy, p.dz = dx, np.full(ny, 0.25), np.full(nz, 1 / 3)
    p.F = np.broadcast_to(Fx, (nz, ny, nx)).copy()
    p.vf = np.ones((nz, ny, nx))
    p.ax = np.broadcast_to(ap, (nz, ny, nx + 1)).copy()
    p.ay, p.az = np.ones((nz, ny + 1, nx)), np.ones((nz + 1, ny, nx))
    p.u = np.broadcast_to(ux, (nz, ny, nx + 1)).copy()
    p.v, p.w = rng.uniform(-1, 1, p.ay.shape) * 0, np.zeros_like(p.az)
    p.rho_liquid, p.rho_gas = 1000.0, 1.2
    p.merge_threshold = 0.0
    s = oracle.System(p)
    ph = s.solve_dense()
    # 1-D: per unit area, conductance between centres i-1, i is a_i / (rho dx/2 + rho dx/2)
    rho = 1.2 + 998.8 * Fx
    half = rho * dx / 2
    c = np.zeros(nx + 1)
    c[1:-1] = ap[1:-1] / (half[:-1] + half[1:])
    c[-1] = ap[-1] / half[-1]            # p = 0 on the x_max face
    main = c[:-1] + c[1:]
    ab = np.zeros((3, nx))
    ab[0, 1:] = -c[1:-1]
    ab[1] = main
    ab[2, :-1] = -c[1:-1]
    flux = ap * ux
    flux[0] = 0.0                        # free-slip x_min wall
    rhs = -(flux[1:] - flux[:-1])
    line = sla.solve_banded((1, 1), ab, rhs)
    np.testing.assert_allclose(ph, np.broadcast_to(line, (nz, ny, nx)), rtol=1e-11, atol=1e-14 * np.abs(line).max())


def test_rhs_is_minus_divergence_closed_form(oracle):
    # u = x on x-faces, zero elsewhere: the outward flux of every cell is its volume, b = -V / dt
    p = I.config1(shape=(16, 8, 8))
    p.bc = (I.DIRICHLET, I.DIRICHLET, I.NEUMANN, I.NEUMANN, I.NEUMANN, I.NEUMANN)
    xn = p.meta["nodes"][0]
    p.vf = np.ones_like(p.vf)
    p.ax, p.ay, p.az = np.ones_like(p.ax), np.ones_like(p.ay), np.ones_like(p.az)
    p.u = np.broadcast_to(xn, p.u.shape).copy()
    p.v, p.w = np.zeros_like(p.v), np.zeros_like(p.w)
    p.dt = 0.5
    b = oracle.rhs(p)
    np.testing.assert_allclose(b, -cell_volumes(p) / 0.5, rtol=1e-13)


def test_all_neumann_nullspace_and_compatibility(oracle):
    p = I.tiny_sphere()
    p.bc = (I.NEUMANN,) * 6
    s = oracle.System(p)
    A = s.Ahat
    ones = np.ones(s.M)
    assert np.abs(A @ ones).max() <= 1e-13 * abs(A).max()
    assert abs(s.bhat.sum()) <= 1e-13 * np.abs(s.bhat).sum()
    x = s.solve_dense()
    assert s.residual(x) < 1e-12


def test_incompatible_all_neumann_rhs_is_an_error(oracle):
    # an all-Neumann right-hand side that does not sum to zero has no solution: the oracle refuses
    # it instead of projecting it onto the compatible subspace
    p = I.tiny_sphere()
    p.bc = (I.NEUMANN,) * 6
    s = oracle.System(p)
    s.bhat = s.bhat + 1e-3 * np.abs(s.bhat).max()
    assert s.compatibility() > 1e-6
    with pytest.raises(ValueError, match="incompatible"):
        s.solve_pcg(rtol=1e-10)
    with pytest.raises(ValueError, match="incompatible"):
        s.solve_dense()


def test_pcg_mark_is_the_same_iterate_as_a_looser_solve(oracle):
    # the iteration at which a tight solve first meets a looser tolerance is the iteration count of
    # a solve to that tolerance (the same iterates), and its time lies inside the whole solve's
    p = I.config1(shape=(32, 16, 16))
    s = oracle.System(p)
    _, loose = s.solve_pcg(rtol=1e-6)
    _, tight = s.solve_pcg(rtol=1e-11, mark_rtol=1e-6)
    assert tight["mark"]["iterations"] == loose["iterations"] > 0
    assert 0.0 < tight["mark"]["seconds"] <= tight["seconds"]
    assert tight["iterations"] > loose["iterations"]


def test_projection_makes_velocity_divergence_free(oracle):
    # Sec. 2.1 Eq. runge1: u* = u - dt (1/rho) grad p; with the solved p every merge group's net
    # outward flux of u* vanishes to solver tolerance.
    p = I.tiny_sphere(n=8)
    p.dt = 0.3
    s = oracle.System(p)
    ph = s.solve_dense()
    nz, ny, nx = p.shape
    rho = oracle.density(p.F, p.rho_liquid, p.rho_gas)
    inactive, ex, ey, ez = (s.inactive, *s.apertures)
    dx, dy, dz = p.dx, p.dy, p.dz
    Sx = (dz[:, None] * dy[None, :])[:, :, None]
    Sy = (dz[:, None] * dx[None, :])[:, None, :]
    Sz = (dy[:, None] * dx[None, :])[None]
    fx = ex * Sx * p.u
    fy = ey * Sy * p.v
    fz = ez * Sz * p.w
    fx[:, :, 0] = 0.0                                         # walls: no normal flux
    fy[:, 0], fy[:, -1], fz[0], fz[-1] = 0.0, 0.0, 0.0, 0.0
    # face gradient of p divided by the face density of the half-cell harmonic average
    fx[:, :, 1:-1] -= p.dt * ex[:, :, 1:-1] * Sx * (ph[:, :, 1:] - ph[:, :, :-1]) / (
        0.5 * (dx[:-1] * rho[:, :, :-1] + dx[1:] * rho[:, :, 1:]))
    fx[:, :, -1] -= p.dt * ex[:, :, -1] * Sx[:, :, 0] * (0.0 - ph[:, :, -1]) / (0.5 * dx[-1] * rho[:, :, -1])
    fy[:, 1:-1, :] -= p.dt * ey[:, 1:-1, :] * Sy * (ph[:, 1:, :] - ph[:, :-1, :]) / (
        0.5 * (dy[:-1, None] * rho[:, :-1, :] + dy[1:, None] * rho[:, 1:, :]))
    fz[1:-1] -= p.dt * ez[1:-1] * Sz * (ph[1:] - ph[:-1]) / (
        0.5 * (dz[:-1, None, None] * rho[:-1] + dz[1:, None, None] * rho[1:]))
    div = (fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:] - fy[:, :-1]) + (fz[1:] - fz[:-1])
    div_groups = s.fold(div)
    scale = np.abs(s.fold((ex * Sx * np.abs(p.u))[:, :, 1:])).max()
    assert np.abs(div_groups).max() <= 1e-12 * scale


def test_projection_functions_give_divergence_free_groups(oracle):
    # oracle.project / oracle.divergence (Sec. 2.1 Eq. runge1) with the dense solution: every
    # merge group's net outward flux vanishes (Dirichlet exit, free-slip walls)
    p = I.tiny_sphere(n=8)
    p.dt = 0.3
    s = oracle.System(p)
    ph = s.solve_dense()
    u, v, w = oracle.project(p, s, ph)
    div = oracle.divergence(p, s, u, v, w)
    ex = s.apertures[0]
    scale = np.abs(s.fold((ex * np.abs(p.u))[:, :, 1:])).max() * p.dx.max() ** 2
    assert np.abs(div).max() <= 1e-12 * scale
    # the unprojected field is far from divergence-free (the check has teeth)
    assert np.abs(oracle.divergence(p, s, p.u, p.v, p.w)).max() > 1e-3 * scale


def test_projection_all_neumann_with_prescribed_wall_flux(oracle):
    # free-slip everywhere, outward (1/rho) dp/dn = g0 on the -x wall and -g0 on the +x wall
    # (compatible: the prescribed fluxes sum to zero); the projected wall velocities are +dt g0
    # and +dt g0 (sign of the outward normal) and every group is divergence-free
    p = I.tiny_sphere(n=8)
    p.dt = 0.7
    p.bc = (0, 0, 0, 0, 0, 0)
    nz, ny, nx = p.shape
    g0 = np.random.default_rng(11).uniform(-1, 1, (nz, ny))
    flux = [g0, -g0, None, None, None, None]
    s = oracle.System(p, neumann_flux=flux)
    assert abs(s.bhat.sum()) <= 1e-12 * np.abs(s.bhat).sum()
    ph = s.solve_dense()
    u, v, w = oracle.project(p, s, ph, neumann_flux=flux)
    np.testing.assert_allclose(u[:, :, 0], p.dt * g0, rtol=1e-15)
    np.testing.assert_allclose(u[:, :, -1], p.dt * g0, rtol=1e-15)
    assert np.all(v[:, 0, :] == 0) and np.all(w[-1] == 0)
    div = oracle.divergence(p, s, u, v, w)
    scale = np.abs(s.fold((s.apertures[0] * np.abs(p.u))[:, :, 1:])).max() * p.dx.max() ** 2
    # the singular all-Neumann system is solved by least squares: about 1e-12 relative accuracy
    assert np.abs(div).max() <= 1e-11 * scale
    assert np.abs(oracle.divergence(p, s, p.u, p.v, p.w)).max() > 1e-3 * scale


def test_exit_flux_of_a_linear_profile_closed_form(oracle):
    # Sec. 2.6 Eq. exit with u = a x + c on the x faces of a stretched grid: du/dx = a exactly, so
    # g = u_c a + R - u_exit / dt on every exit face (the last cell's width, not the first's)
    p = I.tiny_sphere(n=8)
    p.bc = (0, 0, 0, 0, 0, 0)
    p.dt = 0.4
    p.dx = np.array([0.05, 0.07, 0.1, 0.12, 0.14, 0.16, 0.18, 0.18])
    a, c0, uc = 0.73, -0.2, 1.7
    xf = np.concatenate([[0.0], np.cumsum(p.dx)])
    p.u = np.broadcast_to(a * xf + c0, p.u.shape).copy()
    R = np.random.default_rng(2).uniform(-1, 1, p.u.shape[:2])
    g, shift = oracle.exit_flux(p, uc, R=R)
    assert shift == 0.0
    np.testing.assert_allclose(g, uc * a + R - (a * xf[-1] + c0) / p.dt, rtol=1e-12, atol=1e-13)


def test_exit_flux_balance_makes_the_all_neumann_problem_compatible(oracle):
    # the radiation condition alone leaves sum(b_hat) != 0 (Sec. 2.6: it does not conserve mass);
    # the uniform shift over the open exit faces makes the merged system compatible, and a closed
    # exit face keeps its value
    p = I.tiny_sphere(n=8)
    p.bc = (0, 0, 0, 0, 0, 0)
    p.dt = 0.5
    p.ax = p.ax.copy()
    p.ax[0, 0, -1] = 0.0                                        # one closed exit face
    g0, _ = oracle.exit_flux(p, 1.3)
    s0 = oracle.System(p, neumann_flux=[None, g0, None, None, None, None])
    assert abs(s0.bhat.sum()) > 1e-6 * np.abs(s0.bhat).sum()
    g, shift = oracle.exit_flux(p, 1.3, balance=True)
    s = oracle.System(p, neumann_flux=[None, g, None, None, None, None])
    assert abs(s.bhat.sum()) <= 1e-12 * np.abs(s.bhat).sum()
    assert shift != 0.0 and g[0, 0] == g0[0, 0]
    np.testing.assert_allclose((g0 - g)[s.apertures[0][:, :, -1] > 0], shift, rtol=1e-12)


def test_exit_projection_is_the_discrete_orlanski_update(oracle):
    # with the balanced exit flux the all-Neumann solve and the projection (Sec. 2.1 Eq. runge1)
    # give every open exit face u_exit - dt (u_c du/dx + R) + dt * shift, i.e. Eq. orlanski
    # advanced by dt with the momentum balance of Eq. exit, and every merge group is divergence-free
    p = I.tiny_sphere(n=8)
    p.bc = (0, 0, 0, 0, 0, 0)
    p.dt = 0.5
    uc = 0.9
    R = np.random.default_rng(4).uniform(-1, 1, p.u.shape[:2])
    g, shift = oracle.exit_flux(p, uc, R=R, balance=True)
    flux = [None, g, None, None, None, None]
    s = oracle.System(p, neumann_flux=flux)
    ph = s.solve_dense()
    u, v, w = oracle.project(p, s, ph, neumann_flux=flux)
    ue, uu = p.u[:, :, -1], p.u[:, :, -2]
    want = ue - p.dt * (uc * (ue - uu) / p.dx[-1] + R) + p.dt * shift
    open_ = s.apertures[0][:, :, -1] > 0
    np.testing.assert_allclose(u[:, :, -1][open_], want[open_], rtol=1e-12, atol=1e-12)
    div = oracle.divergence(p, s, u, v, w)
    scale = np.abs(s.fold((s.apertures[0] * np.abs(p.u))[:, :, 1:])).max() * p.dx.max() ** 2
    assert np.abs(div).max() <= 1e-11 * scale
    assert np.abs(oracle.divergence(p, s, p.u, p.v, p.w)).max() > 1e-3 * scale


def test_projection_of_a_linear_pressure_closed_form(oracle):
    # uniform grid, rho = 1, p = a x at the cell centres: every open interior x face loses dt*a,
    # y and z faces keep their velocity, and the p = 0 face at x = 1 (half a cell from the last
    # centre) loses dt * (0 - a x_last) / (dx/2)
    n, a, dt = 5, 0.37, 0.6
    p = I.manufactured(n)
    p.dt = dt
    rng = np.random.default_rng(5)
    p.u, p.v, p.w = rng.uniform(-1, 1, p.u.shape), rng.uniform(-1, 1, p.v.shape), rng.uniform(-1, 1, p.w.shape)
    s = oracle.System(p)
    xc = 0.5 * (p.meta["nodes"][0][:-1] + p.meta["nodes"][0][1:])
    pres = np.broadcast_to(a * xc, p.shape)
    u, v, w = oracle.project(p, s, pres)
    np.testing.assert_allclose(u[:, :, 1:-1], p.u[:, :, 1:-1] - dt * a, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[:, :, -1], p.u[:, :, -1] + dt * a * xc[-1] / (0.5 * p.dx[-1]), rtol=1e-14)
    assert np.all(u[:, :, 0] == 0)                           # free-slip wall, no prescribed flux
    np.testing.assert_array_equal(v[:, 1:-1, :], p.v[:, 1:-1, :])
    np.testing.assert_array_equal(w[1:-1], p.w[1:-1])


def test_lanczos_estimates_inside_spectrum(oracle):
    p = I.tiny_sphere()
    s = oracle.System(p)
    _, info = s.solve_pcg(rtol=1e-13, history=True)
    lo, hi = oracle.lanczos_extremes(info["alpha"], info["beta"])
    A = s.Ahat.toarray()
    d = np.diag(A) ** -0.5
    ev = np.linalg.eigvalsh(d[:, None] * A * d)
    assert ev[0] * (1 - 1e-8) <= lo and hi <= ev[-1] * (1 + 1e-8)
    assert hi / lo > 0.5 * ev[-1] / ev[0]


def _handmade(vf, ax=None, ay=None, az=None, threshold=0.1):
    nz, ny, nx = vf.shape
    p = I.manufactured(2)
    p.dx, p.dy, p.dz = np.ones(nx), np.ones(ny), np.ones(nz)
    p.F = np.ones_like(vf)
    p.vf = vf
    p.ax = np.ones((nz, ny, nx + 1)) if ax is None else ax
    p.ay = np.ones((nz, ny + 1, nx)) if ay is None else ay
    p.az = np.ones((nz + 1, ny, nx)) if az is None else az
    p.u, p.v, p.w = np.zeros_like(p.ax), np.zeros_like(p.ay), np.zeros_like(p.az)
    p.merge_threshold = threshold
    return p


def test_merge_goes_to_largest_open_face(oracle):
    vf = np.ones((1, 3, 3))
    vf[0, 1, 1] = 0.05
    ay = np.ones((1, 4, 3))
    ay[0, 2, 1] = 0.7                  # +y face of the centre cell is the largest open one
    ax = np.ones((1, 3, 4)) * 0.5
    ay[0, 1, 1] = 0.3
    p = _handmade(vf, ax=ax, ay=ay)
    s = oracle.System(p)
    assert s.root[4] == 7              # centre (j=1, i=1) -> (j=2, i=1)
    assert (s.root == np.arange(9)).sum() == 8


def test_merge_tie_takes_first_direction(oracle):
    vf = np.ones((1, 1, 3))
    vf[0, 0, 1] = 0.01
    s = oracle.System(_handmade(vf))
    assert s.root[1] == 0              # -x and +x faces tie; -x comes first


def test_merge_chain_and_cycle(oracle):
    # chain: cell 0 (small) -> cell 1 (small) -> cell 2 (large)
    vf = np.array([[[0.02, 0.05, 0.9, 1.0]]])
    ax = np.array([[[1.0, 0.8, 0.9, 0.1, 1.0]]])
    s = oracle.System(_handmade(vf, ax=ax))
    assert list(s.root[:3]) == [2, 2, 2]
    # cycle: two small cells whose largest faces face each other, isolated by closed faces
    vf = np.array([[[1.0, 0.03, 0.06, 1.0]]])
    ax = np.array([[[1.0, 0.1, 0.9, 0.1, 1.0]]])
    s = oracle.System(_handmade(vf, ax=ax))
    assert s.root[1] == 2 and s.root[2] == 2


def test_inactive_cells_and_isolation(oracle):
    vf = np.ones((1, 1, 4))
    vf[0, 0, 2] = 0.0
    ax = np.ones((1, 1, 5))
    ax[0, 0, 1] = 0.0                  # cell 1: open only towards the vf = 0 cell 2
    p = _handmade(vf, ax=ax)
    p.bc = (I.NEUMANN, I.DIRICHLET, I.NEUMANN, I.NEUMANN, I.NEUMANN, I.NEUMANN)
    s = oracle.System(p)
    assert list(s.root) == [-1, -1, -1, 3]   # cell 0 has no open flux face either
