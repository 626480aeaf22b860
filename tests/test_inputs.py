"""Closed-form checks of the seeded input generator (grid stretching, VOF fraction, bodies)."""
import math

import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I


def cell_volumes(p):
    return p.dz[:, None, None] * p.dy[None, :, None] * p.dx[None, None, :]


def test_tanh_nodes_equidistribute_inverse_spacing():
    # Sec. 2.2 Eq. grid: (w x_xi)_xi = 0, so w * dx is the same for every cell with w = 1/h.
    n = 200
    xn = I.tanh_nodes(-1.0, 2.0, n, 0.0, 0.5)
    dx = np.diff(xn)
    xm = 0.5 * (xn[1:] + xn[:-1])
    S = 0.5 * (1 + np.tanh((np.abs(np.linspace(-1, 2, 400001)) - 0.5) / 0.06))
    lo, hi = S.min(), S.max()
    h = 1 + 7 * (0.5 * (1 + np.tanh((np.abs(xm) - 0.5) / 0.06)) - lo) / (hi - lo)
    ratio = dx / h
    assert np.max(np.abs(ratio / ratio.mean() - 1)) < 2e-2
    assert abs(dx.max() / dx.min() - 8.0) < 0.1
    assert xn[0] == -1.0 and xn[-1] == 2.0 and np.all(dx > 0)


def test_flat_surface_fraction():
    zn = np.array([-1.0, -0.25, 0.1, 0.3, 1.0])
    F = I.vof_flat(np.array([0.0, 1.0]), np.array([0.0, 1.0]), zn, 0.2)
    np.testing.assert_allclose(F[:, 0, 0], [1.0, 1.0, 0.5, 0.0], atol=1e-15)


@pytest.mark.parametrize("amp,lam,theta", [(0.05, 1.0, 0.0), (0.02, 0.3, 1.3), (0.011, 0.23, 4.0)])
def test_cosine_surface_water_volume_closed_form(amp, lam, theta):
    # sum F V = integral of (eta - z_bottom) dx * L_y for eta = a cos(2 pi x / lam + theta)
    xn = I.tanh_nodes(-1.0, 2.0, 96, 0.0, 0.5)
    yn = np.linspace(-0.5, 0.5, 3)
    zn = I.tanh_nodes(-1.0, 0.5, 40, 0.0, 0.0625)
    F = I.vof_cosine(xn, yn, zn, amp, lam, theta)
    V = np.diff(zn)[:, None, None] * np.diff(yn)[None, :, None] * np.diff(xn)[None, None, :]
    k = 2 * math.pi / lam
    exact = (amp / k * (math.sin(k * 2.0 + theta) - math.sin(-k + theta)) + 1.0 * 3.0) * 1.0
    assert abs((F * V).sum() - exact) < 1e-13
    assert F.min() >= 0 and F.max() <= 1


def test_cosine_surface_single_cell_brute_force():
    # one cell straddling the crest, fraction by fine midpoint quadrature of clip(eta - z0, 0, dz)
    xn = np.array([-0.07, 0.09])
    zn = np.array([0.01, 0.04])
    F = I.vof_cosine(xn, np.array([0.0, 1.0]), zn, 0.05, 1.0, 0.2)[0, 0, 0]
    xs = np.linspace(-0.07, 0.09, 2000001)
    xm = 0.5 * (xs[1:] + xs[:-1])
    eta = 0.05 * np.cos(2 * np.pi * xm + 0.2)
    ref = np.clip(eta - 0.01, 0, 0.03).mean() / 0.03
    assert abs(F - ref) < 1e-9


def test_sphere_volume():
    p = I.config1(shape=(64, 32, 32))
    blocked = ((1 - p.vf) * cell_volumes(p)).sum()
    assert abs(blocked - 4 / 3 * math.pi * 0.15 ** 3) < 2e-4 * blocked


def test_sphere_apertures_closed_form_on_center_plane():
    # The x-face through the sphere centre sees a disk of radius R; the blocked areas of all
    # faces on that plane add up to pi R^2.
    n = 16
    xn = np.linspace(-0.5, 0.5, n + 1)
    vf, ax, ay, az = I.body_fractions(xn, xn, xn, I.Sphere((0.0, 0.0, 0.0), 0.3))
    S = (1.0 / n) ** 2
    i = n // 2
    assert abs(((1 - ax[:, :, i]) * S).sum() - math.pi * 0.09) < 2e-3 * math.pi * 0.09


def test_hull_panel_mesh_is_closed_and_matches_quadrature():
    hull = I.SlenderHull()
    V, T = hull.triangles()
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    mesh_volume = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert mesh_volume > 0
    # closed mesh: every edge appears twice with opposite orientation
    edges = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    fw = set(map(tuple, edges))
    assert all((e[1], e[0]) in fw for e in map(tuple, edges))
    # the analytic hull volume (8/9) B L T as the panelisation limit
    assert abs(mesh_volume - hull.volume_exact()) < 2e-3 * hull.volume_exact()
    # the grid quadrature of the same body approaches the mesh volume
    p = I.config2(shape=(256, 128, 64))
    blocked = ((1 - p.vf) * cell_volumes(p)).sum()
    assert abs(blocked - mesh_volume) < 5e-3 * mesh_volume


def test_velocities_seeded_and_uniform():
    a = I.config0()
    b = I.config0()
    np.testing.assert_array_equal(a.u, b.u)
    assert a.u.shape == (32, 32, 33) and a.v.shape == (32, 33, 32) and a.w.shape == (33, 32, 32)
    assert -1 <= a.u.min() and a.u.max() <= 1 and abs(a.u.mean()) < 0.02


def test_manufactured_pressure_boundary_conditions():
    p = I.manufactured(8)
    ph = I.manufactured_pressure(p)
    assert ph.shape == (8, 8, 8) and np.all(np.isfinite(ph))
    x = np.linspace(0, 1, 11)
    assert abs(math.cos(0.5 * math.pi * 1.0)) < 1e-15 and x[-1] == 1.0
