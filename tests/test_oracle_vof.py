"""Pins of the VOF oracle (Sec. 2.4: flux-error correction, operator-split advection with
dilation) against closed forms, brute force and conservation (no GPU)."""
import numpy as np
import pytest

from paper_1410_1937_gb300 import inputs as I


@pytest.fixture(scope="module")
def vof():
    from oracle import vof as V
    return V


def quad_volume(m, alpha, h, n=1200):
    # fluid volume below the plane by midpoint quadrature of the clipped fluid height, taken along
    # the axis of the largest normal component (the height is then a gentle function of the rest)
    ax = int(np.argmax(np.abs(m)))
    perm = [i for i in range(3) if i != ax] + [ax]
    m, h = np.asarray(m)[perm], np.asarray(h)[perm]
    x = (np.arange(n) + 0.5) / n * h[0]
    y = (np.arange(n) + 0.5) / n * h[1]
    X, Y = np.meshgrid(x, y, indexing="ij")
    rest = alpha - m[0] * X - m[1] * Y
    if m[2] > 0:
        height = np.clip(rest / m[2], 0.0, h[2])
    elif m[2] < 0:
        height = h[2] - np.clip(rest / m[2], 0.0, h[2])
    else:
        height = np.where(rest >= 0, h[2], 0.0)
    return height.mean() * h[0] * h[1]


def test_box_volume_against_quadrature(vof):
    rng = np.random.default_rng(0)
    for trial in range(24):
        m = rng.normal(size=3)
        if trial % 6 == 1:
            m[rng.integers(3)] = 0.0
        if trial % 6 == 2:
            m[rng.integers(3)] = 1e-9 * np.abs(m).max()
        h = rng.uniform(0.3, 2.0, 3)
        span = np.abs(m * h).sum()
        lo = np.minimum(m * h, 0).sum()
        alpha = lo + rng.uniform(0.02, 0.98) * span
        got = float(vof.box_volume(m, alpha, h))
        assert abs(got - quad_volume(m, alpha, h)) <= 2e-6 * h.prod(), (trial, m, alpha)


def test_box_volume_closed_forms(vof):
    h = np.array([0.7, 1.3, 0.4])
    # horizontal plane: a layer of depth alpha
    for a in (0.0, 0.1, 0.25, 0.4):
        assert abs(vof.box_volume(np.array([0.0, 0.0, 1.0]), a, h) - a * h[0] * h[1]) <= 1e-15
    # complement: {m.x <= a} and {-m.x <= -a} fill the box
    rng = np.random.default_rng(1)
    for _ in range(10):
        m = rng.normal(size=3)
        a = rng.uniform(-1, 1)
        tot = vof.box_volume(m, a, h) + vof.box_volume(-m, -a, h)
        assert abs(tot - h.prod()) <= 1e-14
    # corner tetrahedron: a^3 / (6 m1 m2 m3) while the plane cuts only the corner
    m = np.array([1.0, 2.0, 3.0])
    a = 0.2
    assert abs(vof.box_volume(m, a, h) - a ** 3 / (6 * 6.0)) <= 1e-16


def test_plane_constant_inverts_the_volume(vof):
    rng = np.random.default_rng(2)
    m = rng.normal(size=(50, 3))
    m[::7, 0] = 0.0
    h = rng.uniform(0.3, 2.0, (50, 3))
    phi = rng.uniform(0.0, 1.0, 50)
    a = vof.plane_constant(m, h, phi)
    np.testing.assert_allclose(vof.box_volume(m, a, h), phi * h.prod(axis=1), rtol=0, atol=1e-13)


def test_flux_correction_conserves_each_cell_along_z_only(vof):
    # Sec. 2.4: after the vertical reassignment every cell's own fluxes balance; x and y velocities
    # are the aperture times the velocity; a cell with both z faces closed keeps its fluxes
    p = I.tiny_sphere(n=8)
    ux, uy, wm, wp, E = vof.flux_correct(p)
    dx, dy, dz = p.dx, p.dy, p.dz
    Sx = (dz[:, None] * dy[None, :])[:, :, None]
    Sy = (dz[:, None] * dx[None, :])[:, None, :]
    Sz = (dy[:, None] * dx[None, :])[None, :, :]
    np.testing.assert_allclose(ux, p.ax * p.u, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(uy, p.ay * p.v, rtol=1e-15, atol=1e-15)
    net = (ux[:, :, 1:] - ux[:, :, :-1]) * Sx + (uy[:, 1:] - uy[:, :-1]) * Sy + (wp - wm) * Sz
    closed = (p.az[1:] + p.az[:-1]) == 0
    scale = np.abs(p.ax * Sx * p.u).max()
    assert np.abs(net[~closed]).max() <= 1e-14 * scale
    assert np.abs(E).max() > 1e-3 * scale                      # the input is not solenoidal
    np.testing.assert_array_equal(wp[closed], (p.az * p.w)[1:][closed])
    # the reassignment splits E between the two z faces in proportion to their open areas
    Az = p.az * Sz
    ok = ~closed
    with np.errstate(divide="ignore", invalid="ignore"):
        share = E * Az[1:] / (Az[1:] + Az[:-1])
    np.testing.assert_allclose((((p.az * p.w)[1:] - wp) * Sz)[ok], share[ok], rtol=1e-12, atol=1e-14 * scale)


def plane_fractions(xn, yn, zn, n, d, sub=64):
    # exact-enough fractions of {n.x <= d} per cell by sub-cell sampling of the clipped height
    F = np.zeros((len(zn) - 1, len(yn) - 1, len(xn) - 1))
    from oracle import vof as V
    for k in range(len(zn) - 1):
        for j in range(len(yn) - 1):
            for i in range(len(xn) - 1):
                h = np.array([xn[i + 1] - xn[i], yn[j + 1] - yn[j], zn[k + 1] - zn[k]])
                a = d - n[0] * xn[i] - n[1] * yn[j] - n[2] * zn[k]
                F[k, j, i] = V.box_volume(n, a, h) / h.prod()
    return F


def open_box(n, nx=None):
    nx = nx or n
    xn = np.linspace(0.0, 1.0, nx + 1)
    yn = zn = np.linspace(0.0, 1.0, n + 1)
    z = np.zeros
    p = I.Problem(name="vof-box", dx=np.diff(xn), dy=np.diff(yn), dz=np.diff(zn), F=z((n, n, nx)),
                  vf=np.ones((n, n, nx)), ax=np.ones((n, n, nx + 1)), ay=np.ones((n, n + 1, nx)),
                  az=np.ones((n + 1, n, nx)), u=z((n, n, nx + 1)), v=z((n, n + 1, nx)), w=z((n + 1, n, nx)),
                  rho_liquid=1000.0, rho_gas=1.2, rtol=1e-10)
    return p, (xn, yn, zn)


@pytest.mark.parametrize("normal,vel", [((0.0, 0.0, 1.0), (0.0, 0.0, 0.3)),
                                        ((1.0, 0.0, 0.0), (0.35, 0.0, 0.0)),
                                        ((1.0, 0.0, 1.0), (0.3, 0.0, 0.0))])
def test_uniform_translation_of_a_plane_is_exact(vof, normal, vel):
    # a planar interface carried by a uniform velocity (Courant 0.3-0.35, no dilation since the
    # velocity is uniform): every stage is an exact geometric flux, so the fractions after the
    # step are those of the translated plane (axis-aligned planes and the 45-degree plane, whose
    # weighted central differences give the exact normal direction)
    n = 12
    p, (xn, yn, zn) = open_box(n)
    nrm = np.array(normal) / np.linalg.norm(normal)
    d = 0.47 * nrm.sum() + 0.013
    p.F = plane_fractions(xn, yn, zn, nrm, d)
    h = 1.0 / n
    dt = 1.0 * h
    p.u[:] = vel[0]
    p.v[:] = vel[1]
    p.w[:] = vel[2]
    shift = np.array(vel) * dt
    want = plane_fractions(xn, yn, zn, nrm, d + nrm @ shift)
    for order in (0, 1):
        got = vof.advect(p, dt=dt, order=order)
        # cells away from the domain walls (inflow there takes the boundary cell as donor)
        inner = np.s_[2:-2, 2:-2, 2:-2]
        np.testing.assert_allclose(got[inner], want[inner], rtol=0, atol=1e-12)


def stream_function_flow(p, xn, zn, amp):
    # discretely divergence-free x-z flow vanishing on the walls: u = dpsi/dz, w = -dpsi/dx from a
    # stream function at the cell corners, psi = amp sin^2(pi x) sin^2(pi z)
    psi = amp * np.sin(np.pi * xn)[None, :] ** 2 * np.sin(np.pi * zn)[:, None] ** 2      # (nz+1, nx+1)
    u = (psi[1:, :] - psi[:-1, :]) / np.diff(zn)[:, None]                                  # (nz, nx+1)
    w = -(psi[:, 1:] - psi[:, :-1]) / np.diff(xn)[None, :]                                 # (nz+1, nx)
    p.u = np.broadcast_to(u[:, None, :], p.u.shape).copy()
    p.w = np.broadcast_to(w[:, None, :], p.w.shape).copy()
    p.v[:] = 0.0


def test_solenoidal_flow_needs_no_correction(vof):
    # a discretely divergence-free field has E = 0, so the corrected z velocities are the input's
    n = 10
    p, (xn, yn, zn) = open_box(n)
    stream_function_flow(p, xn, zn, 0.04)
    ux, uy, wm, wp, E = vof.flux_correct(p)
    scale = np.abs(p.u).max() * p.dy[0] * p.dz[0]
    assert np.abs(E).max() <= 1e-15 * scale * 10
    np.testing.assert_allclose(wp, p.w[1:], rtol=0, atol=1e-15)
    np.testing.assert_allclose(wm, p.w[:-1], rtol=0, atol=1e-15)


def test_dilation_keeps_full_and_empty_cells(vof):
    # with a non-uniform solenoidal flow every stage has a velocity divergence along its axis; the
    # dilation term (implicit in the first two stages, explicit in the third) must return a cell
    # that is full (empty) with full (empty) neighbours to exactly 1 (0): a wrong sign, the wrong
    # stage value in the dilation or a mis-selected donor breaks it; the interface moves
    n = 12
    p, (xn, yn, zn) = open_box(n)
    nrm = np.array([0.2, 0.0, 1.0])
    nrm /= np.linalg.norm(nrm)
    p.F = plane_fractions(xn, yn, zn, nrm, 0.52)
    stream_function_flow(p, xn, zn, 0.05)
    dt = 0.45 / (np.abs(p.u).max() / p.dx[0] + np.abs(p.w).max() / p.dz[0])
    # three stages move fluid at most three cells: cells whose 7x7x7 neighbourhood is all full
    # (all empty) must come back exactly full (empty)
    from scipy.ndimage import maximum_filter, minimum_filter
    full = minimum_filter(p.F, size=7, mode="nearest") == 1.0
    empty = maximum_filter(p.F, size=7, mode="nearest") == 0.0
    assert full.sum() > 20 and empty.sum() > 20
    for order in (0, 1):
        got = vof.advect(p, dt=dt, order=order)
        assert np.abs(got[full] - 1.0).max() <= 1e-14
        assert np.abs(got[empty]).max() <= 1e-14
        assert np.abs(got - p.F).max() > 1e-3
        V = (p.dz[:, None, None] * p.dy[None, :, None] * p.dx[None, None, :])
        # operator splitting with dilation conserves volume only approximately
        assert abs((got * V).sum() - (p.F * V).sum()) <= 1e-3 * (p.F * V).sum()


def test_one_dimensional_interface_cell_closed_form(vof):
    # a row of five cells (fractions 1, 1, 1/2, 0, 0; fluid on the left half of the middle cell),
    # u = a x on the x faces, every z face closed (nothing to correct, the y and z stages are
    # idle): the middle cell receives a full slab of thickness u- dt from its left neighbour and
    # sends none, so the x stage gives (1/2 + u- dt/h) / (1 - a dt) when it comes first (implicit
    # dilation) and 1/2 + u- dt/h + (1/2) a dt when it comes last (explicit)
    nx, h = 5, 0.2
    xn = np.arange(nx + 1) * h
    z = np.zeros
    p = I.Problem(name="vof-row", dx=np.full(nx, h), dy=np.array([0.3]), dz=np.array([0.4]),
                  F=np.array([[[1.0, 1.0, 0.5, 0.0, 0.0]]]), vf=np.ones((1, 1, nx)), ax=np.ones((1, 1, nx + 1)),
                  ay=np.ones((1, 2, nx)), az=np.zeros((2, 1, nx)), u=z((1, 1, nx + 1)), v=z((1, 2, nx)),
                  w=z((2, 1, nx)))
    a = 0.6
    p.u[0, 0, :] = a * xn
    dt = 0.4 * h / (a * xn[-1])
    tm = a * xn[2] * dt
    got0 = vof.advect(p, dt=dt, order=0)
    got1 = vof.advect(p, dt=dt, order=1)
    assert abs(got0[0, 0, 2] - (0.5 + tm / h) / (1.0 - a * dt)) <= 1e-15
    assert abs(got1[0, 0, 2] - (0.5 + tm / h + 0.5 * a * dt)) <= 1e-15
