"""Seeded synthetic inputs for the pressure-projection Poisson solve.

This module builds the arrays that the solve consumes and nothing else:

* cell widths along each axis, uniform or stretched.  Stretching follows the 1-D elliptic grid
  equation of Sec. 2.2 (Eq. grid): its first integral says w * dx/dxi is constant, so the spacing
  is proportional to 1/w.  Nodes are placed by equidistributing 1/h for a tanh-shaped spacing h
  whose largest/smallest ratio is 8;
* the exact VOF fraction F of every cell under a flat or cosine free surface (Sec. 2, phi);
* open-area fractions (apertures, the A_i of Sec. 2.4) of every cell face and open-volume
  fractions of every cell cut by an immersed sphere or by a triangle-panelised slender hull
  (Sec. 2.3);
* seeded U[-1,1] face velocities.

It holds none of the solve's arithmetic (no density law, no face coefficients, no divergence, no
merging): the oracle and the CUDA library each implement those from the paper on their own and
consume these arrays.  Every draw comes from numpy's PCG64 generator in a fixed order.

Layouts (numpy C order, x fastest):
    F, vf          (nz, ny, nx)
    ax, u          (nz, ny, nx+1)    x-faces; face i lies between cells i-1 and i
    ay, v          (nz, ny+1, nx)
    az, w          (nz+1, ny, nx)
Boundary kinds are given per domain face in the order -x, +x, -y, +y, -z, +z with
NEUMANN = 0 and DIRICHLET = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from numpy.polynomial.legendre import leggauss

NEUMANN = 0
DIRICHLET = 1

# Density of water and air in kg/m^3 (the two-phase law's end points, Sec. 2 Eq. density).
RHO_LIQUID = 1000.0
RHO_GAS = 1.2


@dataclasses.dataclass
class Problem:
    """One synthetic workload: grid, geometry, fluid fraction, velocities and solve settings."""

    name: str
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    F: np.ndarray
    vf: np.ndarray
    ax: np.ndarray
    ay: np.ndarray
    az: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    bc: tuple = (NEUMANN, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN)
    rho_liquid: float = RHO_LIQUID
    rho_gas: float = RHO_GAS
    merge_threshold: float = 0.1
    density_smoothing: int = 0
    dt: float = 1.0
    rtol: float = 1e-10
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def shape(self):
        return (len(self.dz), len(self.dy), len(self.dx))

    @property
    def n(self):
        return len(self.dx) * len(self.dy) * len(self.dz)


# ----------------------------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------------------------

def uniform_nodes(s0: float, s1: float, n: int) -> np.ndarray:
    return np.linspace(s0, s1, n + 1)


def tanh_nodes(s0: float, s1: float, n: int, center: float, half_width: float,
               ratio: float = 8.0, delta: float | None = None, samples: int = 400001) -> np.ndarray:
    """Nodes whose spacing is proportional to h(s) = 1 + (ratio-1) * S(s).

    S = 1/2 (1 + tanh((|s - center| - half_width) / delta)), rescaled to [0, 1] over the axis, so
    the finest spacing (inside the plateau |s - center| < half_width) and the coarsest differ by
    ``ratio``.  Nodes equidistribute integral(ds / h), i.e. w = 1/h in the first integral
    w * x_xi = const of the grid equation of Sec. 2.2.
    """
    if delta is None:
        delta = 0.02 * (s1 - s0)
    s = np.linspace(s0, s1, samples)
    S = 0.5 * (1.0 + np.tanh((np.abs(s - center) - half_width) / delta))
    S = (S - S.min()) / max(S.max() - S.min(), 1e-300)
    h = 1.0 + (ratio - 1.0) * S
    g = np.concatenate([[0.0], np.cumsum(0.5 * (1.0 / h[1:] + 1.0 / h[:-1]) * np.diff(s))])
    xi = g / g[-1]
    nodes = np.interp(np.linspace(0.0, 1.0, n + 1), xi, s)
    nodes[0], nodes[-1] = s0, s1
    return nodes


# ----------------------------------------------------------------------------------------------
# VOF fraction (exact)
# ----------------------------------------------------------------------------------------------

def vof_flat(xn, yn, zn, z_surface: float) -> np.ndarray:
    """Fraction of each cell below the plane z = z_surface."""
    z0, z1 = zn[:-1], zn[1:]
    col = np.clip((z_surface - z0) / (z1 - z0), 0.0, 1.0)
    return np.broadcast_to(col[:, None, None], (len(zn) - 1, len(yn) - 1, len(xn) - 1)).copy()


def _cos_level_roots(x0, x1, kappa, theta, amp, level, kmax):
    """Roots of amp*cos(kappa*x+theta) = level inside (x0, x1); padded with x1. Shape (m, 2*kmax)."""
    out = np.repeat(x1[:, None], 2 * kmax, axis=1)
    if amp <= 0 or abs(level) >= amp:
        return out
    base = math.acos(level / amp)
    ph0 = kappa * x0 + theta
    ph1 = kappa * x1 + theta
    col = 0
    for b in (base, -base):
        m0 = np.ceil((ph0 - b) / (2 * math.pi))
        for m in range(kmax):
            ph = b + 2 * math.pi * (m0 + m)
            xr = (ph - theta) / kappa
            ok = (ph > ph0) & (ph < ph1)
            out[:, col] = np.where(ok, xr, x1)
            col += 1
    return out


def vof_cosine(xn, yn, zn, amp: float, wavelength: float, phase: float) -> np.ndarray:
    """Exact fraction of each cell below eta(x) = amp*cos(2 pi x / wavelength + phase).

    Per (x-cell, z-cell) the fraction is (1/(dx dz)) * integral over the x-interval of
    clip(eta - z0, 0, dz); the integrand is split at the crossings eta = z0 and eta = z1 and each
    piece is integrated in closed form.  The surface is uniform in y.
    """
    nx, ny, nz = len(xn) - 1, len(yn) - 1, len(zn) - 1
    kappa = 2 * math.pi / wavelength
    x0, x1 = xn[:-1], xn[1:]
    kmax = int(math.ceil(kappa * float(np.max(x1 - x0)) / (2 * math.pi))) + 1
    Fxz = np.zeros((nz, nx))
    for k in range(nz):
        za, zb = zn[k], zn[k + 1]
        if zb <= -amp:
            Fxz[k] = 1.0
            continue
        if za >= amp:
            continue
        pts = np.concatenate([x0[:, None],
                              _cos_level_roots(x0, x1, kappa, phase, amp, za, kmax),
                              _cos_level_roots(x0, x1, kappa, phase, amp, zb, kmax),
                              x1[:, None]], axis=1)
        pts.sort(axis=1)
        xa, xb = pts[:, :-1], pts[:, 1:]
        xm = 0.5 * (xa + xb)
        em = amp * np.cos(kappa * xm + phase)
        mid = (amp / kappa) * (np.sin(kappa * xb + phase) - np.sin(kappa * xa + phase)) - za * (xb - xa)
        piece = np.where(em <= za, 0.0, np.where(em >= zb, (zb - za) * (xb - xa), mid))
        Fxz[k] = np.clip(piece.sum(axis=1) / ((x1 - x0) * (zb - za)), 0.0, 1.0)
    return np.broadcast_to(Fxz[:, None, :], (nz, ny, nx)).copy()


# ----------------------------------------------------------------------------------------------
# Immersed bodies: apertures and open-volume fractions by quadrature
# ----------------------------------------------------------------------------------------------

def _overlap(a0, a1, b0, b1):
    return np.clip(np.minimum(a1, b1) - np.maximum(a0, b0), 0.0, None)


def _gl(n):
    t, wts = leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * wts        # nodes and weights on [0, 1]


def _index_range(nodes, lo, hi):
    """Index range [i0, i1) of cells of a 1-D node array overlapping [lo, hi]."""
    i0 = max(int(np.searchsorted(nodes, lo, side="right")) - 1, 0)
    i1 = min(int(np.searchsorted(nodes, hi, side="left")) + 1, len(nodes) - 1)
    return i0, max(i1, i0)


class Sphere:
    """Ball of radius R centred at c: inside where |x - c| < R."""

    def __init__(self, center, radius):
        self.c = np.asarray(center, dtype=np.float64)
        self.R = float(radius)

    def bbox(self):
        return self.c - self.R, self.c + self.R

    def cell_blocked(self, X0, X1, Y0, Y1, Z0, Z1, q=8):
        """Blocked volume fraction: 2-D Gauss-Legendre in (x, y), exact z-chord length."""
        t, wq = _gl(q)
        frac = 0.0
        for a in range(q):
            xs = X0 + (X1 - X0) * t[a]
            for b in range(q):
                ys = Y0 + (Y1 - Y0) * t[b]
                H = np.sqrt(np.clip(self.R ** 2 - (xs - self.c[0]) ** 2 - (ys - self.c[1]) ** 2, 0.0, None))
                frac = frac + wq[a] * wq[b] * _overlap(Z0, Z1, self.c[2] - H, self.c[2] + H) / (Z1 - Z0)
        return frac

    def face_blocked(self, axis, P, A0, A1, B0, B1, q=16):
        """Blocked area fraction of the face at coordinate P on ``axis``; (A, B) are the other two
        axes in increasing order.  1-D Gauss-Legendre along A, exact chord along B."""
        ia, ib = [d for d in range(3) if d != axis]
        t, wq = _gl(q)
        frac = 0.0
        for a in range(q):
            As = A0 + (A1 - A0) * t[a]
            H = np.sqrt(np.clip(self.R ** 2 - (P - self.c[axis]) ** 2 - (As - self.c[ia]) ** 2, 0.0, None))
            frac = frac + wq[a] * _overlap(B0, B1, self.c[ib] - H, self.c[ib] + H) / (B1 - B0)
        return frac

    def volume(self):
        return 4.0 / 3.0 * math.pi * self.R ** 3


class SlenderHull:
    """Panelised slender hull |y - y0| < h_PL(x - x0, z - z0).

    The analytic half-beam is h(x, z) = (B/2)(1 - (2x/L)^2)(1 - (z/T)^2) on |x| <= L/2, |z| <= T,
    zero on the rim, so the surface y = +-h closes.  It is panelised on an (x, z) parameter grid of
    ``panels`` quads, two triangles per quad, on each side y = +h and y = -h.  The body enclosed by
    that triangle mesh is exactly {|y - y0| < h_PL} where h_PL interpolates h linearly on those
    triangles, so inside tests need no ray casting.
    """

    def __init__(self, origin=(0.0, 0.0, 0.0), L=1.0, B=0.1, T=0.0625, panels=(256, 64)):
        self.o = np.asarray(origin, dtype=np.float64)
        self.L, self.B, self.T = float(L), float(B), float(T)
        self.npx, self.npz = panels
        xs = np.linspace(-self.L / 2, self.L / 2, self.npx + 1)
        zs = np.linspace(-self.T, self.T, self.npz + 1)
        self.hn = (self.B / 2) * (1 - (2 * xs[:, None] / self.L) ** 2) * (1 - (zs[None, :] / self.T) ** 2)
        self.hn[0, :] = 0.0
        self.hn[-1, :] = 0.0
        self.hn[:, 0] = 0.0
        self.hn[:, -1] = 0.0

    def bbox(self):
        lo = self.o + np.array([-self.L / 2, -self.B / 2, -self.T])
        hi = self.o + np.array([self.L / 2, self.B / 2, self.T])
        return lo, hi

    def half_beam(self, X, Z):
        """h_PL at body-relative (X, Z); zero outside the parameter rectangle."""
        X = np.asarray(X, dtype=np.float64)
        Z = np.asarray(Z, dtype=np.float64)
        uu = (X + self.L / 2) / (self.L / self.npx)
        ww = (Z + self.T) / (2 * self.T / self.npz)
        inside = (uu > 0) & (uu < self.npx) & (ww > 0) & (ww < self.npz)
        i = np.clip(np.floor(uu).astype(np.int64), 0, self.npx - 1)
        j = np.clip(np.floor(ww).astype(np.int64), 0, self.npz - 1)
        fu = np.clip(uu - i, 0.0, 1.0)
        fw = np.clip(ww - j, 0.0, 1.0)
        h00 = self.hn[i, j]
        h10 = self.hn[i + 1, j]
        h01 = self.hn[i, j + 1]
        h11 = self.hn[i + 1, j + 1]
        lower = fu + fw <= 1.0
        hl = h00 + fu * (h10 - h00) + fw * (h01 - h00)
        hu = h11 + (1.0 - fu) * (h01 - h11) + (1.0 - fw) * (h10 - h11)
        return np.where(inside, np.where(lower, hl, hu), 0.0)

    def triangles(self):
        """Vertex (V, 3) and triangle (T, 3) arrays of the closed panelisation, outward oriented."""
        xs = np.linspace(-self.L / 2, self.L / 2, self.npx + 1)
        zs = np.linspace(-self.T, self.T, self.npz + 1)
        XX, ZZ = np.meshgrid(xs, zs, indexing="ij")
        nv = XX.size
        verts = []
        for sgn in (+1.0, -1.0):
            verts.append(np.stack([XX.ravel(), sgn * self.hn.ravel(), ZZ.ravel()], axis=1))
        V = np.concatenate(verts) + self.o
        idx = np.arange(nv).reshape(self.npx + 1, self.npz + 1)
        a = idx[:-1, :-1].ravel()
        b = idx[1:, :-1].ravel()
        c = idx[:-1, 1:].ravel()
        d = idx[1:, 1:].ravel()
        # +y side: normal must point to +y; (x, z) -> (b - a) x (c - a) = ex x ez = -ey, so flip.
        plus = np.concatenate([np.stack([a, c, b], 1), np.stack([d, b, c], 1)])
        # the -y side reuses the rim vertices (h = 0 there) so that the mesh is closed
        rim = np.zeros((self.npx + 1, self.npz + 1), dtype=bool)
        rim[0, :] = rim[-1, :] = rim[:, 0] = rim[:, -1] = True
        remap = np.where(rim.ravel(), np.arange(nv), np.arange(nv) + nv)
        minus = remap[np.concatenate([np.stack([a, b, c], 1), np.stack([d, c, b], 1)])]
        return V, np.concatenate([plus, minus])

    def volume_exact(self):
        return 8.0 / 9.0 * self.B * self.L * self.T

    def cell_blocked(self, X0, X1, Y0, Y1, Z0, Z1, q=8):
        t, wq = _gl(q)
        frac = 0.0
        for a in range(q):
            xs = X0 + (X1 - X0) * t[a]
            for b in range(q):
                zs = Z0 + (Z1 - Z0) * t[b]
                H = self.half_beam(xs - self.o[0], zs - self.o[2])
                frac = frac + wq[a] * wq[b] * _overlap(Y0, Y1, self.o[1] - H, self.o[1] + H) / (Y1 - Y0)
        return frac

    def face_blocked(self, axis, P, A0, A1, B0, B1, q=16):
        if axis == 1:
            # plane y = P: blocked where h_PL(x, z) > |P - y0|; midpoint sampling in (x, z)
            s = (np.arange(q) + 0.5) / q
            c = np.abs(P - self.o[1])
            frac = 0.0
            for a in range(q):
                xs = A0 + (A1 - A0) * s[a]
                for b in range(q):
                    zs = B0 + (B1 - B0) * s[b]
                    frac = frac + (self.half_beam(xs - self.o[0], zs - self.o[2]) > c)
            return frac / (q * q)
        t, wq = _gl(q)
        frac = 0.0
        for a in range(q):
            if axis == 0:        # plane x = P; A = y carries the chord, integrate along B = z
                zs = B0 + (B1 - B0) * t[a]
                H = self.half_beam(P - self.o[0], zs - self.o[2])
                frac = frac + wq[a] * _overlap(A0, A1, self.o[1] - H, self.o[1] + H) / (A1 - A0)
            else:                # plane z = P; integrate along A = x, chord along B = y
                xs = A0 + (A1 - A0) * t[a]
                H = self.half_beam(xs - self.o[0], P - self.o[2])
                frac = frac + wq[a] * _overlap(B0, B1, self.o[1] - H, self.o[1] + H) / (B1 - B0)
        return frac


def body_fractions(xn, yn, zn, body):
    """Open-volume fractions vf and face apertures (ax, ay, az) of the grid around ``body``.

    Cells and faces outside the body's bounding box are fully open.  Inside it the blocked fraction
    comes from the body's quadrature; results are clipped to [0, 1] and values within 1e-12 of 0 or
    1 are snapped so that fully covered and fully open cells are exact.
    """
    nx, ny, nz = len(xn) - 1, len(yn) - 1, len(zn) - 1
    vf = np.ones((nz, ny, nx))
    ax = np.ones((nz, ny, nx + 1))
    ay = np.ones((nz, ny + 1, nx))
    az = np.ones((nz + 1, ny, nx))
    lo, hi = body.bbox()
    i0, i1 = _index_range(xn, lo[0], hi[0])
    j0, j1 = _index_range(yn, lo[1], hi[1])
    k0, k1 = _index_range(zn, lo[2], hi[2])
    if i1 <= i0 or j1 <= j0 or k1 <= k0:
        return vf, ax, ay, az

    def snap(a):
        a = np.clip(a, 0.0, 1.0)
        a[a < 1e-12] = 0.0
        a[a > 1 - 1e-12] = 1.0
        return a

    X0 = xn[i0:i1][None, :]
    X1 = xn[i0 + 1:i1 + 1][None, :]
    Y0 = yn[j0:j1][:, None]
    Y1 = yn[j0 + 1:j1 + 1][:, None]
    for k in range(k0, k1):
        Z0, Z1 = zn[k], zn[k + 1]
        vf[k, j0:j1, i0:i1] = snap(1.0 - body.cell_blocked(X0, X1, Y0, Y1, Z0, Z1))
        # x-faces of this z-layer at nodes xn[i0 .. i1]
        P = xn[i0:i1 + 1][None, :]
        ax[k, j0:j1, i0:i1 + 1] = snap(1.0 - body.face_blocked(0, P, Y0, Y1, Z0, Z1))
        # y-faces at nodes yn[j0 .. j1]
        Py = yn[j0:j1 + 1][:, None]
        ay[k, j0:j1 + 1, i0:i1] = snap(1.0 - body.face_blocked(1, Py, X0, X1, Z0, Z1))
    for k in range(k0, k1 + 1):
        ax_ = xn[i0:i1][None, :]
        az[k, j0:j1, i0:i1] = snap(1.0 - body.face_blocked(2, zn[k], ax_, X1, Y0, Y1))
    return vf, ax, ay, az


# ----------------------------------------------------------------------------------------------
# Velocities and workloads
# ----------------------------------------------------------------------------------------------

def face_velocities(rng: np.random.Generator, nx: int, ny: int, nz: int):
    u = rng.uniform(-1.0, 1.0, size=(nz, ny, nx + 1))
    v = rng.uniform(-1.0, 1.0, size=(nz, ny + 1, nx))
    w = rng.uniform(-1.0, 1.0, size=(nz + 1, ny, nx))
    return u, v, w


def _assemble(name, xn, yn, zn, F, body, rng, **kw):
    nx, ny, nz = len(xn) - 1, len(yn) - 1, len(zn) - 1
    if body is None:
        vf = np.ones((nz, ny, nx))
        ax = np.ones((nz, ny, nx + 1))
        ay = np.ones((nz, ny + 1, nx))
        az = np.ones((nz + 1, ny, nx))
    else:
        vf, ax, ay, az = body_fractions(xn, yn, zn, body)
    u, v, w = face_velocities(rng, nx, ny, nz)
    meta = kw.pop("meta", {})
    meta.update(nodes=(xn, yn, zn))
    return Problem(name=name, dx=np.diff(xn), dy=np.diff(yn), dz=np.diff(zn), F=F, vf=vf,
                   ax=ax, ay=ay, az=az, u=u, v=v, w=w, meta=meta, **kw)


def hull_domain_nodes(nx, ny, nz):
    """Domain 3 x 1 x 1.5 ship lengths (x in [-1, 2], y in [-1/2, 1/2], z in [-1, 1/2]) with
    cells clustered on the hull's length, beam and draft (Sec. 3, Athena domain proportions)."""
    xn = tanh_nodes(-1.0, 2.0, nx, 0.0, 0.5)
    yn = tanh_nodes(-0.5, 0.5, ny, 0.0, 0.05)
    zn = tanh_nodes(-1.0, 0.5, nz, 0.0, 0.0625)
    return xn, yn, zn


def config0(seed: int = 0, n: int = 32) -> Problem:
    """32^3 uniform cells on [-1/2, 1/2]^3, surface 0.05 cos(2 pi x), no body, p = 0 at x_max."""
    xn = yn = zn = uniform_nodes(-0.5, 0.5, n)
    F = vof_cosine(xn, yn, zn, 0.05, 1.0, 0.0)
    rng = np.random.default_rng(seed)
    return _assemble(f"uniform-{n}^3-cosine-wave", xn, yn, zn, F, None, rng, rtol=1e-10)


def config1(seed: int = 1, shape=(128, 64, 64)) -> Problem:
    """Stretched 128x64x64 grid on [-1,1]x[-1/2,1/2]^2 around a half-immersed sphere r = 0.15."""
    nx, ny, nz = shape
    xn = tanh_nodes(-1.0, 1.0, nx, 0.0, 0.15)
    yn = tanh_nodes(-0.5, 0.5, ny, 0.0, 0.15)
    zn = tanh_nodes(-0.5, 0.5, nz, 0.0, 0.15)
    F = vof_flat(xn, yn, zn, 0.0)
    rng = np.random.default_rng(seed)
    body = Sphere((0.0, 0.0, 0.0), 0.15)
    return _assemble(f"sphere-{nx}x{ny}x{nz}", xn, yn, zn, F, body, rng, rtol=1e-10,
                     meta={"body": body})


def _hull_wave_problem(name, shape, rng, origin, amp, lam, theta, rtol):
    nx, ny, nz = shape
    xn, yn, zn = hull_domain_nodes(nx, ny, nz)
    F = vof_cosine(xn, yn, zn, amp, lam, theta)
    body = SlenderHull(origin)
    return _assemble(name, xn, yn, zn, F, body, rng, rtol=rtol,
                     meta={"body": body, "wave": (amp, lam, theta), "origin": tuple(origin)})


def config2(seed: int = 2, shape=(512, 256, 128)) -> Problem:
    """Slender hull in random waves on the 3 x 1 x 1.5 domain, 512x256x128 stretched cells."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2 * math.pi)
    amp = rng.uniform(0.005, 0.02)
    lam = rng.uniform(0.2, 0.5)
    nx, ny, nz = shape
    return _hull_wave_problem(f"hull-waves-{nx}x{ny}x{nz}", shape, rng, (0.0, 0.0, 0.0),
                              amp, lam, theta, 1e-8)


def config3_sample(seed: int, shape=(256, 128, 64)) -> Problem:
    """Training/held-out sample: hull offset, waves and velocities all drawn from ``seed``."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-0.2, 0.2)
    y0 = rng.uniform(-0.1, 0.1)
    z0 = rng.uniform(-0.01, 0.01)
    theta = rng.uniform(0.0, 2 * math.pi)
    amp = rng.uniform(0.005, 0.02)
    lam = rng.uniform(0.2, 0.5)
    nx, ny, nz = shape
    return _hull_wave_problem(f"hull-sample{seed}-{nx}x{ny}x{nz}", shape, rng, (x0, y0, z0),
                              amp, lam, theta, 1e-10)


def config4(seed: int = 4, shape=(1024, 512, 256)) -> Problem:
    """Steep wave (a = 0.03, wavelength 0.25) around the slender hull, 1024x512x256 cells."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2 * math.pi)
    nx, ny, nz = shape
    return _hull_wave_problem(f"hull-steep-{nx}x{ny}x{nz}", shape, rng, (0.0, 0.0, 0.0),
                              0.03, 0.25, theta, 1e-8)


def config(i: int, **kw) -> Problem:
    return (config0, config1, config2, lambda **k: config3_sample(200000, **k), config4)[i](**kw)


def momentum_terms(prob: Problem, seed: int = 21):
    """Seeded stand-in for the momentum terms R of Sec. 2.1 (convection, hydrostatics, viscosity,
    sub-grid and body forces) on the x, y and z faces: independent U[-1, 1] values."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, prob.u.shape), rng.uniform(-1.0, 1.0, prob.v.shape),
            rng.uniform(-1.0, 1.0, prob.w.shape))


def tiny_sphere(n: int = 8, seed: int = 7, radius: float = 0.3, threshold: float = 0.25,
                center=(0.05, -0.02, 0.03)) -> Problem:
    """n^3 uniform cells on [-1/2,1/2]^3 cut by a sphere, with merging; small enough for dense
    linear algebra."""
    xn = yn = zn = uniform_nodes(-0.5, 0.5, n)
    F = vof_cosine(xn, yn, zn, 0.08, 0.7, 0.3)
    rng = np.random.default_rng(seed)
    body = Sphere(center, radius)
    p = _assemble(f"tiny-sphere-{n}^3", xn, yn, zn, F, body, rng, rtol=1e-12, meta={"body": body})
    p.merge_threshold = threshold
    return p


def manufactured(n: int) -> Problem:
    """Uniform n^3 grid on [0,1]^3, constant density 1, no body, p = 0 at x = 1.  The right-hand
    side is set later from the closed-form pressure (velocities are zero)."""
    xn = yn = zn = uniform_nodes(0.0, 1.0, n)
    z = np.zeros
    p = Problem(name=f"manufactured-{n}^3", dx=np.diff(xn), dy=np.diff(yn), dz=np.diff(zn),
                F=np.ones((n, n, n)), vf=np.ones((n, n, n)), ax=np.ones((n, n, n + 1)),
                ay=np.ones((n, n + 1, n)), az=np.ones((n + 1, n, n)), u=z((n, n, n + 1)),
                v=z((n, n + 1, n)), w=z((n + 1, n, n)), rho_liquid=1.0, rho_gas=1.0, rtol=1e-12,
                meta={"nodes": (xn, yn, zn)})
    return p


def manufactured_pressure(prob: Problem) -> np.ndarray:
    """p = cos(pi x / 2) cos(pi y) cos(pi z) at cell centres: zero normal derivative on x = 0 and on
    the y, z walls, p = 0 at x = 1, and -lap p = (9 pi^2 / 4) p."""
    xn, yn, zn = prob.meta["nodes"]
    xc = 0.5 * (xn[1:] + xn[:-1])
    yc = 0.5 * (yn[1:] + yn[:-1])
    zc = 0.5 * (zn[1:] + zn[:-1])
    return (np.cos(np.pi * zc / 1.0)[:, None, None] * np.cos(np.pi * yc)[None, :, None]
            * np.cos(0.5 * np.pi * xc)[None, None, :])


def manufactured_rhs(prob: Problem) -> np.ndarray:
    """Cell-integrated source V_c * (1/rho) * (9 pi^2 / 4) * p(x_c) for the closed form above."""
    V = prob.dz[:, None, None] * prob.dy[None, :, None] * prob.dx[None, None, :]
    return V * (9.0 * np.pi ** 2 / 4.0) * manufactured_pressure(prob) / prob.rho_liquid
