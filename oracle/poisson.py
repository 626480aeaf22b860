"""Oracle: plain, slow FP64 CPU reference of the pressure-projection Poisson solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package.  The product (``paper_1410_1937_gb300.vofp``
and ``libvofp.so``) never calls it, and it shares no code with the CUDA path: it reads the same
seeded input arrays and nothing else.

What it computes is the unique solution of the discrete finite-volume pressure equation, written
out from its definition:

* density of each cell from its VOF fraction, rho = rho_g + (rho_l - rho_g) F, i.e. the two-phase
  law rho = lambda + (1 - lambda) H(phi) of Sec. 2 (Eq. density) with H(phi) = phi in dimensional
  units; optional (1/4, 1/2, 1/4) smoothing along each axis in turn (Sec. 2.10);
* the integral form of the Poisson equation over each cell's open faces (Sec. 2.3, Eqs.
  integral1 and integral2): the flux through a face is aperture x area x (p_R - p_L) / (half-cell
  resistance sum), i.e. T_f = A_f S_f / ((d_L rho_L + d_R rho_R) / 2); a face with p = 0 on it
  (Dirichlet) gets T = A S / (d_c rho_c / 2) on the diagonal; free-slip faces carry no flux
  (Sec. 1; Sec. 2.3);
* the right-hand side -(1/dt) * sum of outward face fluxes A_f S_f u_f (Sec. 2.1 Eq. poisson1 and
  Sec. 2.4, F_i = A_i (u_i - v_i)), plus the body-surface term of Eq. integral2 and prescribed
  outward pressure fluxes on Neumann faces (Sec. 2.6, Eq. exit), both optional;
* the exit flux of the radiation condition (Sec. 2.6, Eqs. orlanski and exit), optionally shifted
  uniformly over the open exit faces so that the all-Neumann problem is compatible;
* merging of cells whose open volume is below a threshold (Sec. 2.3) as the explicit triple
  product P^T A P, one unknown per merge group;
* the solution of that system by textbook Jacobi-PCG (oracle/pcg.c) to a tight tolerance, or by
  dense LU on tiny grids.

The assembly loops over faces (each face adds +-T to two rows of a sparse matrix), unlike the
CUDA path's cell-centred stencil.  Readings of points the paper leaves open are listed with each
function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import time

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

NEUMANN, DIRICHLET = 0, 1


# ----------------------------------------------------------------------------------------------
# Build / load the C part
# ----------------------------------------------------------------------------------------------

def build(force: bool = False) -> str:
    """Compile oracle/pcg.c into oracle/_build/liboracle_pcg.so with gcc (OpenMP)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liboracle_pcg.so")
    src = os.path.join(_HERE, "pcg.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o", so + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(so + ".tmp", so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        i64, dp, ip64, ip32 = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), \
            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
        lib.oracle_jacobi_pcg.restype = ctypes.c_int
        lib.oracle_jacobi_pcg.argtypes = [i64, ip64, ip32, dp, dp, dp, ctypes.c_double, i64,
                                          ip64, dp, dp, dp, ctypes.c_double, ip64, dp]
        lib.oracle_csr_matvec.restype = None
        lib.oracle_csr_matvec.argtypes = [i64, ip64, ip32, dp, dp, dp]
        lib.oracle_set_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _LIB = lib
    return _LIB


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count of the C part (0 = leave as is); returns the count in use."""
    return _lib().oracle_set_threads(int(n))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ----------------------------------------------------------------------------------------------
# Cells: density and activity
# ----------------------------------------------------------------------------------------------

def density(F, rho_l, rho_g, smoothing=False):
    """rho = rho_g + (rho_l - rho_g) F (Sec. 2 Eq. density, H(phi) = phi).  With smoothing, the
    three-point (1/4, 1/2, 1/4) filter of Sec. 2.10 runs along x, then y, then z; at a domain wall
    the missing neighbour is replaced by the cell itself."""
    rho = rho_g + (rho_l - rho_g) * np.asarray(F, dtype=np.float64)
    if smoothing:
        for axis in (2, 1, 0):
            lo = np.concatenate([np.take(rho, [0], axis), np.take(rho, np.arange(rho.shape[axis] - 1), axis)], axis)
            hi = np.concatenate([np.take(rho, np.arange(1, rho.shape[axis]), axis),
                                 np.take(rho, [rho.shape[axis] - 1], axis)], axis)
            rho = 0.25 * lo + 0.5 * rho + 0.25 * hi
    return rho


def activity(vf, ax, ay, az, bc):
    """Inactive cells and the apertures that remain after removing them.

    Reading: a cell has no unknown when its open volume is zero, or when none of its faces that
    can carry pressure flux (interior faces and p = 0 domain faces) is open.  Every face of an
    inactive cell is closed (A = 0 inside the hull, Sec. 2.4); closing faces can isolate further
    cells, so the rule is applied until nothing changes.
    """
    nz, ny, nx = vf.shape
    inactive = ~(vf > 0.0)
    while True:
        ex, ey, ez = ax.copy(), ay.copy(), az.copy()
        ex[:, :, 1:] *= ~inactive
        ex[:, :, :-1] *= ~inactive
        ey[:, 1:, :] *= ~inactive
        ey[:, :-1, :] *= ~inactive
        ez[1:, :, :] *= ~inactive
        ez[:-1, :, :] *= ~inactive
        # faces that may carry flux: interior faces, and domain faces whose kind is Dirichlet
        open_x = ex > 0
        open_y = ey > 0
        open_z = ez > 0
        for arr, axis, (lo_kind, hi_kind) in ((open_x, 2, bc[0:2]), (open_y, 1, bc[2:4]), (open_z, 0, bc[4:6])):
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[axis] = 0
            sl_hi[axis] = arr.shape[axis] - 1
            if lo_kind != DIRICHLET:
                arr[tuple(sl_lo)] = False
            if hi_kind != DIRICHLET:
                arr[tuple(sl_hi)] = False
        has_open = (open_x[:, :, :-1] | open_x[:, :, 1:] | open_y[:, :-1, :] | open_y[:, 1:, :]
                    | open_z[:-1, :, :] | open_z[1:, :, :])
        new_inactive = inactive | ~has_open
        if np.array_equal(new_inactive, inactive):
            return inactive, ex, ey, ez
        inactive = new_inactive


# ----------------------------------------------------------------------------------------------
# Assembly of the unmerged operator and right-hand side
# ----------------------------------------------------------------------------------------------

def _cell_index(shape):
    nz, ny, nx = shape
    return np.arange(nz * ny * nx, dtype=np.int64).reshape(nz, ny, nx)


def assemble(prob, F=None):
    """Unmerged operator A (CSR, N x N) and the merge-independent pieces it needs.

    Per interior face between cells L and R along an axis with cell widths d_L, d_R, open fraction
    A_f and full face area S_f:  T_f = A_f S_f / ((d_L rho_L + d_R rho_R) / 2)  (the face
    coefficient 1/rho averaged harmonically with half-cell distance weights, times aperture times
    area over distance; Sec. 2.3 Eq. integral2).  A gets +T at (L,L) and (R,R), -T at (L,R) and
    (R,L).  A domain face with p = 0 on it adds A_f S_f / (d_c rho_c / 2) to (c,c).
    """
    nz, ny, nx = prob.shape
    N = nx * ny * nz
    rho = density(prob.F if F is None else F, prob.rho_liquid, prob.rho_gas, bool(prob.density_smoothing))
    inactive, ex, ey, ez = activity(prob.vf, prob.ax, prob.ay, prob.az, prob.bc)
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    idx = _cell_index(prob.shape)
    rows, cols, vals = [], [], []
    diag_extra = np.zeros(N)

    def add_faces(Tf, L, R):
        Tf, L, R = Tf.ravel(), L.ravel(), R.ravel()
        keep = Tf != 0
        Tf, L, R = Tf[keep], L[keep], R[keep]
        rows.extend([L, R, L, R])
        cols.extend([L, R, R, L])
        vals.extend([Tf, Tf, -Tf, -Tf])

    # x faces: interior faces i = 1 .. nx-1 between cells i-1 and i
    Sx = (dz[:, None] * dy[None, :])[:, :, None]
    dL = dx[None, None, :-1]
    dR = dx[None, None, 1:]
    Tx = ex[:, :, 1:-1] * Sx / (0.5 * (dL * rho[:, :, :-1] + dR * rho[:, :, 1:]))
    add_faces(Tx, idx[:, :, :-1], idx[:, :, 1:])
    Sy = (dz[:, None] * dx[None, :])[:, None, :]
    dL = dy[None, :-1, None]
    dR = dy[None, 1:, None]
    Ty = ey[:, 1:-1, :] * Sy / (0.5 * (dL * rho[:, :-1, :] + dR * rho[:, 1:, :]))
    add_faces(Ty, idx[:, :-1, :], idx[:, 1:, :])
    Sz = (dy[:, None] * dx[None, :])[None, :, :]
    dL = dz[:-1, None, None]
    dR = dz[1:, None, None]
    Tz = ez[1:-1, :, :] * Sz / (0.5 * (dL * rho[:-1, :, :] + dR * rho[1:, :, :]))
    add_faces(Tz, idx[:-1, :, :], idx[1:, :, :])

    # Dirichlet domain faces (p = 0 on the face, half a cell from the centre)
    bc = prob.bc
    if bc[0] == DIRICHLET:
        diag_extra[idx[:, :, 0].ravel()] += (ex[:, :, 0] * Sx[:, :, 0] / (0.5 * dx[0] * rho[:, :, 0])).ravel()
    if bc[1] == DIRICHLET:
        diag_extra[idx[:, :, -1].ravel()] += (ex[:, :, -1] * Sx[:, :, 0] / (0.5 * dx[-1] * rho[:, :, -1])).ravel()
    if bc[2] == DIRICHLET:
        diag_extra[idx[:, 0, :].ravel()] += (ey[:, 0, :] * Sy[:, 0, :] / (0.5 * dy[0] * rho[:, 0, :])).ravel()
    if bc[3] == DIRICHLET:
        diag_extra[idx[:, -1, :].ravel()] += (ey[:, -1, :] * Sy[:, 0, :] / (0.5 * dy[-1] * rho[:, -1, :])).ravel()
    if bc[4] == DIRICHLET:
        diag_extra[idx[0].ravel()] += (ez[0] * Sz[0] / (0.5 * dz[0] * rho[0])).ravel()
    if bc[5] == DIRICHLET:
        diag_extra[idx[-1].ravel()] += (ez[-1] * Sz[0] / (0.5 * dz[-1] * rho[-1])).ravel()

    r = np.concatenate(rows + [np.arange(N)])
    c = np.concatenate(cols + [np.arange(N)])
    v = np.concatenate(vals + [diag_extra])
    A = sp.coo_matrix((v, (r, c)), shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A, inactive, (ex, ey, ez)


def rhs(prob, apertures=None, body_flux=None, neumann_flux=None):
    """Per-cell right-hand side b_c = -(1/dt) (sum_f sigma_f A_f S_f u_f + body_flux_c)
    + sum over Neumann domain faces of A_f S_f g_f.

    sigma_f = +1 on a cell's + face, -1 on its - face (outward flux; Sec. 2.4 F_i = A_i u_i).
    Normal velocities on free-slip domain faces are not used (they are zero at a wall); those on
    p = 0 faces are.  ``body_flux`` is the integral of v*.n over the cell's body surface (Sec. 2.3
    Eq. integral2); ``neumann_flux[f]`` the prescribed outward (1/rho) dp/dn on domain face f
    (Sec. 2.6 Eq. exit).  Cells without an unknown get 0.
    """
    if apertures is None:
        inactive, ex, ey, ez = activity(prob.vf, prob.ax, prob.ay, prob.az, prob.bc)
    else:
        inactive, ex, ey, ez = apertures
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    bc = prob.bc
    fx = ex * (dz[:, None] * dy[None, :])[:, :, None] * prob.u
    fy = ey * (dz[:, None] * dx[None, :])[:, None, :] * prob.v
    fz = ez * (dy[:, None] * dx[None, :])[None, :, :] * prob.w
    fx = fx.copy(); fy = fy.copy(); fz = fz.copy()
    if bc[0] != DIRICHLET: fx[:, :, 0] = 0.0
    if bc[1] != DIRICHLET: fx[:, :, -1] = 0.0
    if bc[2] != DIRICHLET: fy[:, 0, :] = 0.0
    if bc[3] != DIRICHLET: fy[:, -1, :] = 0.0
    if bc[4] != DIRICHLET: fz[0] = 0.0
    if bc[5] != DIRICHLET: fz[-1] = 0.0
    div = (fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :]) + (fz[1:] - fz[:-1])
    if body_flux is not None:
        div = div + body_flux
    b = -div / prob.dt
    if neumann_flux is not None:
        Sx = (dz[:, None] * dy[None, :])
        Sy = (dz[:, None] * dx[None, :])
        Sz = (dy[:, None] * dx[None, :])
        g = neumann_flux
        if g[0] is not None and bc[0] == NEUMANN: b[:, :, 0] += ex[:, :, 0] * Sx * g[0]
        if g[1] is not None and bc[1] == NEUMANN: b[:, :, -1] += ex[:, :, -1] * Sx * g[1]
        if g[2] is not None and bc[2] == NEUMANN: b[:, 0, :] += ey[:, 0, :] * Sy * g[2]
        if g[3] is not None and bc[3] == NEUMANN: b[:, -1, :] += ey[:, -1, :] * Sy * g[3]
        if g[4] is not None and bc[4] == NEUMANN: b[0] += ez[0] * Sz * g[4]
        if g[5] is not None and bc[5] == NEUMANN: b[-1] += ez[-1] * Sz * g[5]
    b[inactive] = 0.0
    return b


# ----------------------------------------------------------------------------------------------
# Merging (Sec. 2.3)
# ----------------------------------------------------------------------------------------------

def merge_roots(prob, inactive, apertures):
    """Root (master) cell of every cell; -1 for cells without an unknown.

    Reading of Sec. 2.3: an active cell whose open volume fraction is below the threshold merges
    with the neighbour across its interior face of largest open area A_f S_f (first of -x, +x, -y,
    +y, -z, +z on ties); a small cell with no open interior face stays alone.  Chains are followed
    until a cell that does not merge; a cycle of small cells is rooted at its member of largest
    open volume (lowest index on ties).
    """
    ex, ey, ez = apertures
    nz, ny, nx = prob.shape
    N = nx * ny * nz
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    vf = prob.vf.ravel()
    act = ~inactive.ravel()
    small = act & (vf < prob.merge_threshold)
    Sx = (dz[:, None] * dy[None, :])[:, :, None]
    Sy = (dz[:, None] * dx[None, :])[:, None, :]
    Sz = (dy[:, None] * dx[None, :])[None, :, :]
    areas = np.zeros((6, nz, ny, nx))
    areas[0, :, :, 1:] = (ex * Sx)[:, :, 1:-1]       # -x face of cells i >= 1
    areas[1, :, :, :-1] = (ex * Sx)[:, :, 1:-1]      # +x face of cells i <= nx-2
    areas[2, :, 1:, :] = (ey * Sy)[:, 1:-1, :]
    areas[3, :, :-1, :] = (ey * Sy)[:, 1:-1, :]
    areas[4, 1:, :, :] = (ez * Sz)[1:-1]
    areas[5, :-1, :, :] = (ez * Sz)[1:-1]
    areas = areas.reshape(6, N)
    offs = np.array([-1, 1, -nx, nx, -nx * ny, nx * ny])
    target = {}
    for c in np.nonzero(small)[0]:
        a = areas[:, c]
        f = int(np.argmax(a))
        if a[f] > 0.0:
            target[int(c)] = int(c + offs[f])
    root_of = {}

    def resolve(c):
        path, pos, cur = [], {}, c
        while True:
            if cur in root_of:
                r = root_of[cur]
                break
            if cur not in target:
                r = cur
                break
            if cur in pos:
                cyc = path[pos[cur]:]
                r = max(cyc, key=lambda m: (vf[m], -m))
                for m in cyc:
                    root_of[m] = r
                break
            pos[cur] = len(path)
            path.append(cur)
            cur = target[cur]
        for m in path:
            root_of.setdefault(m, r)

    for c in sorted(target):
        resolve(c)
    root = np.where(act, np.arange(N), -1)
    for c, r in root_of.items():
        root[c] = r
    return root


class System:
    """The merged system A_hat p_hat = b_hat on the active merge groups."""

    def __init__(self, prob, body_flux=None, neumann_flux=None):
        self.prob = prob
        t0 = time.perf_counter()
        A, inactive, ap = assemble(prob)
        self.inactive = inactive
        self.apertures = ap
        self.root = merge_roots(prob, inactive, ap)
        N = prob.n
        act = self.root >= 0
        self.masters = np.nonzero(self.root == np.arange(N))[0]
        M = len(self.masters)
        col = np.full(N, -1, dtype=np.int64)
        col[self.masters] = np.arange(M)
        cells = np.nonzero(act)[0]
        # P copies each group's unknown to all its cells: P[c, col(root(c))] = 1
        self.P = sp.csr_matrix((np.ones(len(cells)), (cells, col[self.root[cells]])), shape=(N, M))
        self.A = A
        self.Ahat = (self.P.T @ A @ self.P).tocsr()
        self.Ahat.sum_duplicates()
        self.Ahat.sort_indices()
        self.b = rhs(prob, (inactive, *ap), body_flux, neumann_flux).ravel()
        self.bhat = self.P.T @ self.b
        self.dirichlet = any(k == DIRICHLET for k in prob.bc)
        self.assembly_seconds = time.perf_counter() - t0

    @property
    def M(self):
        return len(self.masters)

    def expand(self, xhat):
        return (self.P @ xhat).reshape(self.prob.shape)

    def restrict(self, x_full):
        return np.asarray(x_full, dtype=np.float64).ravel()[self.masters]

    def fold(self, y_full):
        return self.P.T @ np.asarray(y_full, dtype=np.float64).ravel()

    def apply_full(self, x_full):
        """y = A_hat x_hat with x_hat the masters' values of x; returned on the full grid with the
        group's value at its master and 0 at other cells."""
        y = np.zeros(self.prob.n)
        y[self.masters] = self.Ahat @ self.restrict(x_full)
        return y.reshape(self.prob.shape)

    def residual(self, p_full):
        """||b_hat - A_hat p_hat|| / ||b_hat|| for a full-grid pressure (masters' values used)."""
        ph = self.restrict(p_full)
        bn = np.linalg.norm(self.bhat)
        return np.linalg.norm(self.bhat - self.Ahat @ ph) / (bn if bn > 0 else 1.0)

    def solve_dense(self):
        Ad = self.Ahat.toarray()
        if self.dirichlet:
            ph = np.linalg.solve(Ad, self.bhat)
        else:
            c = self.compatibility()
            if not c <= 1e-12:
                raise ValueError(f"incompatible all-Neumann right-hand side: |sum b| / sum |b| = {c:.3e}")
            ph = np.linalg.lstsq(Ad, self.bhat, rcond=None)[0]
            ph -= ph.mean()
        return self.expand(ph)

    def compatibility(self):
        """|sum of b_hat| relative to sum of |b_hat|: the integral form (Sec. 2.3) over the whole
        domain makes the net outward flux vanish when every boundary is free-slip, so an
        all-Neumann problem has a solution only when this is at rounding level."""
        tot = np.abs(self.bhat).sum()
        return abs(self.bhat.sum()) / tot if tot > 0 else 0.0

    def solve_pcg(self, rtol=1e-12, maxit=200000, x0=None, history=False, mark_rtol=None):
        """Jacobi-PCG (oracle/pcg.c) to ``rtol``.  ``mark_rtol``: also report the iteration and the
        seconds at which the updated residual first met that looser tolerance (info["mark"])."""
        lib = _lib()
        Ah = self.Ahat
        ip = Ah.indptr.astype(np.int64)
        ix = Ah.indices.astype(np.int32)
        a = np.ascontiguousarray(Ah.data, dtype=np.float64)
        b = np.ascontiguousarray(self.bhat, dtype=np.float64)
        if not self.dirichlet:
            # All-Neumann: only a compatible right-hand side has a solution (reading 11 of the
            # integral form); an incompatible one is an error, not something to project away.
            # What remains of a compatible one is rounding, removed with the constant null space.
            c = self.compatibility()
            if not c <= 1e-12:
                raise ValueError(f"incompatible all-Neumann right-hand side: |sum b| / sum |b| = {c:.3e}")
            b = b - b.mean()
        x = np.zeros(self.M) if x0 is None else self.restrict(x0).copy()
        it = ctypes.c_int64(0)
        rr = ctypes.c_double(0.0)
        ah = np.zeros(maxit) if history else None
        bh = np.zeros(maxit) if history else None
        mi = ctypes.c_int64(-1)
        ms = ctypes.c_double(-1.0)
        want_mark = mark_rtol is not None
        t0 = time.perf_counter()
        st = lib.oracle_jacobi_pcg(self.M, _ptr(ip, ctypes.c_int64), _ptr(ix, ctypes.c_int32),
                                   _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double),
                                   _ptr(x, ctypes.c_double), float(rtol), int(maxit),
                                   ctypes.byref(it), ctypes.byref(rr),
                                   _ptr(ah, ctypes.c_double) if history else None,
                                   _ptr(bh, ctypes.c_double) if history else None,
                                   float(mark_rtol) if want_mark else 0.0,
                                   ctypes.byref(mi) if want_mark else None,
                                   ctypes.byref(ms) if want_mark else None)
        secs = time.perf_counter() - t0
        if not self.dirichlet:
            x -= x.mean()
        info = {"status": int(st), "iterations": int(it.value), "rel_residual": float(rr.value),
                "seconds": secs, "threads": set_threads(0)}
        if want_mark:
            info["mark"] = {"rtol": float(mark_rtol), "iterations": int(mi.value), "seconds": float(ms.value)}
        if history:
            n = int(it.value)
            info["alpha"] = ah[:n]
            info["beta"] = bh[:n]
        return self.expand(x), info


# ----------------------------------------------------------------------------------------------
# Projection (Sec. 2.1, Eq. runge1: u = u* - dt (1/rho) grad p) and its divergence check
# ----------------------------------------------------------------------------------------------

def project(prob, s, p_full, neumann_flux=None):
    """Face velocities after the projection u = u* - dt (1/rho) dp/dn on every face, with the
    face's 1/rho and distance those of the operator (half-cell harmonic average, Sec. 2.3):

    * interior face with an open effective aperture: u - dt (p_R - p_L) / ((d_L rho_L + d_R rho_R)/2);
    * p = 0 domain face (open): the outside value is 0 at half a cell, u - dt (p_out - p_in) with
      the distance d_c rho_c / 2, signs following the axis;
    * free-slip domain face: the wall velocity is not used by the right-hand side (it is taken as
      0); with a prescribed outward flux g = (1/rho) dp/dn the projected velocity is -dt g on a +
      face and +dt g on a - face, else 0;
    * a face whose effective aperture is 0 keeps u (no flux passes it).

    ``p_full`` is the full-grid pressure (every cell of a merge group holds the group's value,
    0 where there is no unknown).  Returns (u, v, w) with the shapes of prob.u, prob.v, prob.w.
    """
    ex, ey, ez = s.apertures
    rho = density(prob.F, prob.rho_liquid, prob.rho_gas, bool(prob.density_smoothing))
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    dt = prob.dt
    p = np.asarray(p_full, dtype=np.float64).reshape(prob.shape)
    bc = prob.bc
    g = neumann_flux if neumann_flux is not None else [None] * 6
    u = np.array(prob.u, dtype=np.float64)
    v = np.array(prob.v, dtype=np.float64)
    w = np.array(prob.w, dtype=np.float64)
    # interior faces
    gx = (p[:, :, 1:] - p[:, :, :-1]) / (0.5 * (dx[:-1] * rho[:, :, :-1] + dx[1:] * rho[:, :, 1:]))
    u[:, :, 1:-1] = np.where(ex[:, :, 1:-1] > 0, u[:, :, 1:-1] - dt * gx, u[:, :, 1:-1])
    gy = (p[:, 1:, :] - p[:, :-1, :]) / (0.5 * (dy[:-1, None] * rho[:, :-1, :] + dy[1:, None] * rho[:, 1:, :]))
    v[:, 1:-1, :] = np.where(ey[:, 1:-1, :] > 0, v[:, 1:-1, :] - dt * gy, v[:, 1:-1, :])
    gz = (p[1:] - p[:-1]) / (0.5 * (dz[:-1, None, None] * rho[:-1] + dz[1:, None, None] * rho[1:]))
    w[1:-1] = np.where(ez[1:-1] > 0, w[1:-1] - dt * gz, w[1:-1])

    # domain faces: (array, aperture, face slice, adjacent cell slice, cell width, sign of outward normal)
    def wall(arr, ap, fsl, csl, width, sign, kind, flux):
        if kind == DIRICHLET:
            pin = p[csl]
            grad = sign * (0.0 - pin) / (0.5 * width * rho[csl])   # (p_out - p_in) along +axis
            arr[fsl] = np.where(ap[fsl] > 0, arr[fsl] - dt * grad, arr[fsl])
        else:
            arr[fsl] = 0.0 if flux is None else -sign * dt * flux

    wall(u, ex, np.s_[:, :, 0], np.s_[:, :, 0], dx[0], -1, bc[0], g[0])
    wall(u, ex, np.s_[:, :, -1], np.s_[:, :, -1], dx[-1], +1, bc[1], g[1])
    wall(v, ey, np.s_[:, 0, :], np.s_[:, 0, :], dy[0], -1, bc[2], g[2])
    wall(v, ey, np.s_[:, -1, :], np.s_[:, -1, :], dy[-1], +1, bc[3], g[3])
    wall(w, ez, np.s_[0], np.s_[0], dz[0], -1, bc[4], g[4])
    wall(w, ez, np.s_[-1], np.s_[-1], dz[-1], +1, bc[5], g[5])
    return u, v, w


def exit_flux(prob, u_c, R=None, balance=False, body_flux=None, neumann_flux=None):
    """Prescribed outward flux g = (1/rho) dp/dx on the +x domain face from the radiation condition
    (Sec. 2.6): du/dt + u_c du/dx = 0 (Eq. orlanski) in the x-momentum balance gives
    (1/rho) dp/dx = u_c du/dx + R (Eq. exit).  du/dx is the difference of the x-face velocities
    at the exit face and one cell upstream over the last cell's width.  The free-slip reading of
    the projection sets the projected velocity of a + face to -dt g, so the exit face's own
    velocity enters as -u_exit/dt: the projected exit velocity is then u_exit - dt (u_c du/dx + R).

    With ``balance`` the same amount is subtracted on every open exit face so that the cell
    right-hand sides (rhs with this flux and the other prescribed ones) sum to zero, the condition
    of the all-Neumann problem.  Returns (g with shape (nz, ny), the amount subtracted).
    """
    u = np.asarray(prob.u, dtype=np.float64)
    ue, uu = u[:, :, -1], u[:, :, -2]
    g = u_c * (ue - uu) / prob.dx[-1] - ue / prob.dt
    if R is not None:
        g = g + np.asarray(R, dtype=np.float64).reshape(g.shape)
    shift = 0.0
    if balance:
        inactive, ex, ey, ez = activity(prob.vf, prob.ax, prob.ay, prob.az, prob.bc)
        flux = list(neumann_flux) if neumann_flux is not None else [None] * 6
        flux[1] = g
        b = rhs(prob, (inactive, ex, ey, ez), body_flux, flux)
        Sx = prob.dz[:, None] * prob.dy[None, :]
        area = (ex[:, :, -1] * Sx).sum()
        if area > 0:
            shift = b.sum() / area
            g = np.where(ex[:, :, -1] > 0, g - shift, g)
    return g, shift


def divergence(prob, s, u, v, w, body_flux=None):
    """Net outward flux of the face velocities through each cell's open faces, sum_f sigma_f A_f
    S_f u_f (+ the body-surface flux), folded over merge groups: the group's total at its master,
    0 at its other cells and where there is no unknown (full-grid shape)."""
    ex, ey, ez = s.apertures
    dx, dy, dz = prob.dx, prob.dy, prob.dz
    fx = ex * (dz[:, None] * dy[None, :])[:, :, None] * u
    fy = ey * (dz[:, None] * dx[None, :])[:, None, :] * v
    fz = ez * (dy[:, None] * dx[None, :])[None, :, :] * w
    div = (fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :]) + (fz[1:] - fz[:-1])
    if body_flux is not None:
        div = div + np.asarray(body_flux).reshape(prob.shape)
    out = np.zeros(prob.n)
    out[s.masters] = s.fold(div)
    return out.reshape(prob.shape)


def lanczos_extremes(alpha, beta):
    """Extreme eigenvalues of the Jacobi-preconditioned operator estimated from the CG
    coefficients (the Lanczos tridiagonal matrix that CG builds implicitly)."""
    k = len(alpha)
    if k == 0:
        return float("nan"), float("nan")
    d = np.empty(k)
    e = np.empty(max(k - 1, 0))
    for i in range(k):
        d[i] = 1.0 / alpha[i] + (beta[i - 1] / alpha[i - 1] if i > 0 else 0.0)
        if i < k - 1:
            e[i] = np.sqrt(max(beta[i], 0.0)) / alpha[i]
    from scipy.linalg import eigvalsh_tridiagonal
    ev = eigvalsh_tridiagonal(d, e)
    return float(ev[0]), float(ev[-1])


def solve(prob, rtol=1e-12, dense=None):
    """Full-grid pressure of ``prob`` (masters' values copied to their groups, 0 where there is no
    unknown) and an info dict."""
    sysm = System(prob)
    if dense is None:
        dense = sysm.M <= 4096
    if dense:
        t0 = time.perf_counter()
        p = sysm.solve_dense()
        info = {"status": 0, "iterations": 0, "rel_residual": sysm.residual(p),
                "seconds": time.perf_counter() - t0, "threads": 1}
    else:
        p, info = sysm.solve_pcg(rtol=rtol)
    info["assembly_seconds"] = sysm.assembly_seconds
    return p, info, sysm


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
