"""Oracle: plain FP64 CPU reference of the VOF operator of Sec. 2.4 (flux-error correction and
operator-split advection with dilation), for small grids.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this module; the product never calls it and shares no code with it.

What it computes, in the paper's order:

* face fluxes F_i = A_i (u_i - v_i) (Sec. 2.4): the relative face velocity times the open face
  area (aperture x face area); the relative velocity is the input;
* the conservation error of each cell, E = sum_i (F+_i - F-_i) (Eq. diverge), removed along the
  vertical axis: F~+_3 = F+_3 - E A+_3 / (A+_3 + A-_3), F~-_3 = F-_3 + E A-_3 / (A+_3 + A-_3);
  the corrected z fluxes belong to the cell (the two cells of a z face may disagree);
* the velocities u^_i = dx_i F~_i / V on the uncut faces (x and y faces shared, z faces per cell);
* three operator-split stages, each an advection of the volume fraction through the uncut faces
  with the piecewise-linear interface of the donor cell plus a dilation term: the first two stages
  take the dilation with the stage's new value (implicit), the third with the value before it
  (explicit), as the stage equations print them; the order of the axes alternates between
  (x, y, z) and (z, y, x) from one time step to the next.

Readings where the paper is silent or garbled (each listed in the design notes): the third stage
advects phi~~ (the printed phi^ is not defined); the interface normal is minus the gradient of phi
by central differences weighted (1, 2, 1) x (1, 2, 1) across the other two axes (Youngs), with
neighbours inside the body (no open volume) and outside the domain replaced by the cell itself;
the plane constant makes the fluid volume below the plane equal phi times the cell volume; a cell
with phi in {0, 1} or a zero gradient moves phi times the slab volume; inflow through a domain face
takes the boundary cell as donor (zero gradient of phi at the boundary); a slab is at most the
donor cell; no clipping of phi; a cell whose z faces are both closed is not corrected.
"""
from __future__ import annotations

import numpy as np

AXES = {0: "x", 1: "y", 2: "z"}


# ----------------------------------------------------------------------------------------------
# Fluid volume below a plane inside a box (unit-cube reduction with sorted normal components)
# ----------------------------------------------------------------------------------------------

def unit_fraction(c, beta):
    """Volume of {y in [0,1]^3 : c . y <= beta} for c >= 0 with sum(c) = 1 (rows of c), beta in
    [0, 1].  Region by region, in forms without cancellation when a component is small."""
    c = np.sort(np.asarray(c, dtype=np.float64), axis=-1)
    beta = np.asarray(beta, dtype=np.float64)
    flip = beta > 0.5
    b = np.where(flip, 1.0 - beta, beta)
    c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2]
    c12 = c1 + c2
    out = np.zeros(np.broadcast(b, c1).shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        # corner cut (b < c1): b^3 / (6 c1 c2 c3)
        r1 = b * (b / c1) * b / (6.0 * c2 * c3)
        # wedge (c1 <= b < c2)
        r2 = (b * (b - c1) + c1 * c1 / 3.0) / (2.0 * c2 * c3)
        # two corners cut (c2 <= b < min(c12, c3)): [b^3 - (b-c1)^3 - (b-c2)^3] / (6 c1 c2 c3)
        d2 = b - c2
        p1 = 3.0 * b * b - 3.0 * b * c1 + c1 * c1
        r3 = (p1 - d2 * (d2 / c1) * d2) / (6.0 * c2 * c3)
        # three corners cut (c3 <= b < c12)
        d3 = b - c3
        r4 = (p1 - d2 * (d2 / c1) * d2 - d3 * (d3 / c1) * d3) / (6.0 * c2 * c3)
        # slab through the cube (c12 <= b, b <= c3)
        r5 = (2.0 * b - c12) / (2.0 * c3)
    m3 = np.minimum(c12, c3)
    out = np.where(b < c1, r1,
          np.where(b < c2, r2,
          np.where(b < m3, r3,
          np.where(c3 < c12, r4, r5))))
    out = np.where(b <= 0.0, 0.0, out)
    return np.where(flip, 1.0 - out, out)


def box_volume(m, alpha, h):
    """Volume of {x in [0,h1]x[0,h2]x[0,h3] : m . x <= alpha} (arrays broadcast on the leading
    axes; m and h have a last axis of 3)."""
    m = np.asarray(m, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    neg = m < 0
    # x_i -> h_i - x_i for negative components
    alpha = alpha - np.sum(np.where(neg, m * h, 0.0), axis=-1)
    a = np.abs(m) * h
    s = a.sum(axis=-1)
    vol = h.prod(axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        frac = unit_fraction(a / s[..., None], np.clip(alpha / s, 0.0, 1.0))
    frac = np.where(s > 0, frac, (alpha >= 0).astype(np.float64))
    frac = np.where(alpha <= 0, 0.0, np.where(alpha >= s, 1.0, frac))
    return frac * vol


def plane_constant(m, h, phi, iters=200):
    """alpha with box_volume(m, alpha, h) = phi * prod(h), by bisection on the monotone volume."""
    m = np.asarray(m, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    lo = np.sum(np.minimum(m * h, 0.0), axis=-1)
    hi = np.sum(np.maximum(m * h, 0.0), axis=-1)
    target = np.asarray(phi, dtype=np.float64) * h.prod(axis=-1)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = box_volume(m, mid, h) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


# ----------------------------------------------------------------------------------------------
# Flux-error correction (Sec. 2.4)
# ----------------------------------------------------------------------------------------------

def flux_correct(prob, u=None, v=None, w=None):
    """Face fluxes F = A (u - v), the cell error E and the corrected velocities u^ on the uncut
    faces.  Returns (ux^ (nz, ny, nx+1), uy^ (nz, ny+1, nx), wm^, wp^ (nz, ny, nx): the cell's
    -z and +z face, E (nz, ny, nx))."""
    u = prob.u if u is None else u
    v = prob.v if v is None else v
    w = prob.w if w is None else w
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    Sx = (dz[:, None] * dy[None, :])[:, :, None]
    Sy = (dz[:, None] * dx[None, :])[:, None, :]
    Sz = (dy[:, None] * dx[None, :])[None, :, :]
    Ax, Ay, Az = prob.ax * Sx, prob.ay * Sy, prob.az * Sz
    Fx, Fy, Fz = Ax * u, Ay * v, Az * w
    E = (Fx[:, :, 1:] - Fx[:, :, :-1]) + (Fy[:, 1:, :] - Fy[:, :-1, :]) + (Fz[1:] - Fz[:-1])
    Ap, Am = Az[1:], Az[:-1]
    tot = Ap + Am
    with np.errstate(divide="ignore", invalid="ignore"):
        fp = np.where(tot > 0, Fz[1:] - E * Ap / tot, Fz[1:])
        fm = np.where(tot > 0, Fz[:-1] + E * Am / tot, Fz[:-1])
    # u^_i = dx_i F~_i / V = F~_i / (uncut face area)
    return Fx / Sx, Fy / Sy, fm / Sz, fp / Sz, E


# ----------------------------------------------------------------------------------------------
# Interface reconstruction and one advection stage
# ----------------------------------------------------------------------------------------------

def _centres(d):
    return np.concatenate([[0.0], np.cumsum(d)])[:-1] + 0.5 * d


def normals(phi, prob):
    """m = -grad(phi) per cell (nz, ny, nx, 3 with components x, y, z): central differences over
    the centres of the two neighbours along the axis (a missing neighbour's centre is the cell's
    own centre shifted by its width), weighted (1, 2, 1) x (1, 2, 1) over the other two axes."""
    nz, ny, nx = phi.shape
    P = np.pad(phi, 1, mode="constant")
    O = np.pad(prob.vf > 0, 1, mode="constant")
    val = {}
    for dk in range(3):
        for dj in range(3):
            for di in range(3):
                nb = P[dk:dk + nz, dj:dj + ny, di:di + nx]
                ok = O[dk:dk + nz, dj:dj + ny, di:di + nx]
                val[dk, dj, di] = np.where(ok, nb, phi)
    def span(d):
        c = _centres(d)
        cp = np.concatenate([[c[0] - d[0]], c, [c[-1] + d[-1]]])
        return cp[2:] - cp[:-2]
    wts = (1.0, 2.0, 1.0)
    gx = sum(wts[a] * wts[b] * (val[a, b, 2] - val[a, b, 0]) for a in range(3) for b in range(3)) / 16.0
    gy = sum(wts[a] * wts[b] * (val[a, 2, b] - val[a, 0, b]) for a in range(3) for b in range(3)) / 16.0
    gz = sum(wts[a] * wts[b] * (val[2, a, b] - val[0, a, b]) for a in range(3) for b in range(3)) / 16.0
    gx = gx / span(prob.dx)[None, None, :]
    gy = gy / span(prob.dy)[None, :, None]
    gz = gz / span(prob.dz)[:, None, None]
    return np.stack([-gx, -gy, -gz], axis=-1)


def _slab_volume(phi, m, alpha, h, axis, plus, t):
    """Fluid in the slab of thickness t (at most the cell) at the + or - face of the cell along
    `axis`, from the cell's plane; phi times the slab volume where there is no interface."""
    t = np.minimum(t, h[..., axis])
    hs = h.copy()
    hs[..., axis] = t
    a = alpha - (m[..., axis] * (h[..., axis] - t) if plus else 0.0)
    full = hs.prod(axis=-1)
    interface = (phi > 0.0) & (phi < 1.0) & (np.abs(m).sum(axis=-1) > 0)
    vol = np.where(interface, box_volume(m, a, hs), phi * full)
    return np.where(t > 0, vol, 0.0)


def stage(phi, prob, axis, up, um, dt, implicit, dil_phi=None):
    """One split stage along `axis`: phi_new = phi - (F[u^+] - F[u^-]) / V + dt phi_d (u^+ - u^-)
    / dx_axis, phi_d = phi_new (implicit) or dil_phi (explicit; default phi).  up, um: the
    cell's u^ on its + and - face along the axis (nz, ny, nx)."""
    nz, ny, nx = phi.shape
    h = np.stack(np.broadcast_arrays(prob.dx[None, None, :], prob.dy[None, :, None], prob.dz[:, None, None]),
                 axis=-1).astype(np.float64)
    vol = h.prod(axis=-1)
    m = normals(phi, prob)
    alpha = plane_constant(m, h, phi)
    # neighbour along the axis (the boundary cell itself outside the domain)
    def shift(a, s):
        idx = [slice(None)] * 3
        ax = 2 - axis
        n = a.shape[ax]
        order = np.clip(np.arange(n) + s, 0, n - 1)
        idx[ax] = order
        return a[tuple(idx)]
    hd = h[..., axis]
    # + face: u^+ > 0 moves fluid out of this cell's + slab, u^+ < 0 brings the neighbour's - slab
    own_p = _slab_volume(phi, m, alpha, h, axis, True, np.abs(up) * dt)
    nb_phi, nb_m, nb_a, nb_h = shift(phi, +1), shift(m, +1), shift(alpha, +1), shift(h, +1)
    nb_m_p = _slab_volume(nb_phi, nb_m, nb_a, nb_h, axis, False, np.abs(up) * dt)
    Fp = np.where(up > 0, own_p, -nb_m_p)
    # - face: u^- > 0 brings the -neighbour's + slab in, u^- < 0 moves this cell's - slab out
    own_m = _slab_volume(phi, m, alpha, h, axis, False, np.abs(um) * dt)
    pv_phi, pv_m, pv_a, pv_h = shift(phi, -1), shift(m, -1), shift(alpha, -1), shift(h, -1)
    nb_p_m = _slab_volume(pv_phi, pv_m, pv_a, pv_h, axis, True, np.abs(um) * dt)
    Fm = np.where(um > 0, nb_p_m, -own_m)
    adv = phi - (Fp - Fm) / vol
    div = dt * (up - um) / hd
    if implicit:
        return adv / (1.0 - div)
    base = phi if dil_phi is None else dil_phi
    return adv + base * div


def advect(prob, phi=None, dt=None, order=0, u=None, v=None, w=None):
    """phi^{k+1} = phi^k - VOF(u, phi^k, dt): the flux-error correction, then three split stages
    (axes x, y, z for order 0, z, y, x for order 1), the first two with implicit dilation and the
    third explicit."""
    phi = np.asarray(prob.F if phi is None else phi, dtype=np.float64)
    dt = prob.dt if dt is None else dt
    ux, uy, wm, wp, _ = flux_correct(prob, u, v, w)
    faces = {0: (ux[:, :, 1:], ux[:, :, :-1]), 1: (uy[:, 1:, :], uy[:, :-1, :]), 2: (wp, wm)}
    axes = (0, 1, 2) if order == 0 else (2, 1, 0)
    cur = phi
    for s, a in enumerate(axes):
        up, um = faces[a]
        cur = stage(cur, prob, a, up, um, dt, implicit=(s < 2))
    return cur
