"""Thin ctypes binding of libvofp (include/vofp.h).  Argument marshalling only: every step of the
solve runs in the library's CUDA kernels.  Importing this module fails loudly when libvofp.so has
not been built (``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU fallback.

Module-level functions carry the C names (vofp_create, vofp_build_operator, ...) and take torch
CUDA tensors (float64, contiguous) where the C call takes device pointers; ``Context`` wraps them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvofp.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libvofp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_STAGNATED, \
    ERR_INCOMPATIBLE_RHS, ERR_NOT_BUILT, ERR_DEVICE_TIMEOUT = range(10)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
                6: "STAGNATED", 7: "INCOMPATIBLE_RHS", 8: "NOT_BUILT", 9: "DEVICE_TIMEOUT"}
BC_NEUMANN, BC_DIRICHLET = 0, 1
MODE_FP64, MODE_MIXED, MODE_FCG_NN = 0, 1, 2
PRECOND_JACOBI, PRECOND_RBSGS = 0, 1


class VofpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"vofp status {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double)),
                ("dz", ctypes.POINTER(ctypes.c_double))]


class _Bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("neumann_flux", ctypes.c_void_p * 6)]


class _Phys(ctypes.Structure):
    _fields_ = [("rho_liquid", ctypes.c_double), ("rho_gas", ctypes.c_double),
                ("merge_threshold", ctypes.c_double), ("density_smoothing", ctypes.c_int),
                ("dt", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("precond", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("x0_zero", ctypes.c_int), ("host_loop", ctypes.c_int),
                ("nn", ctypes.c_void_p), ("stag_window", ctypes.c_int), ("inner_restart", ctypes.c_int),
                ("stag_ratio", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("status", ctypes.c_int), ("nn_applications", ctypes.c_int), ("fell_back", ctypes.c_int)]


class _HostStep(ctypes.Structure):
    _fields_ = [("F", ctypes.c_void_p), ("ax", ctypes.c_void_p), ("ay", ctypes.c_void_p), ("az", ctypes.c_void_p),
                ("vol_frac", ctypes.c_void_p), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("x_host", ctypes.c_void_p)]


class _Rk2Info(ctypes.Structure):
    _fields_ = [("solve1", _Info), ("solve2", _Info), ("max_div", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_longlong), ("unknowns", ctypes.c_longlong),
                ("inactive", ctypes.c_longlong), ("merged_cells", ctypes.c_longlong),
                ("groups", ctypes.c_longlong), ("device_bytes", ctypes.c_longlong),
                ("tma_stencil_fp32", ctypes.c_int), ("tma_stencil_fp64", ctypes.c_int), ("rb_compact", ctypes.c_int),
                ("pdl_chained", ctypes.c_int)]


_vp = ctypes.c_void_p
_P = ctypes.POINTER
_sig = {
    "vofp_version": (ctypes.c_char_p, []),
    "vofp_create": (ctypes.c_int, [_P(_vp), _P(_Grid), _vp]),
    "vofp_destroy": (None, [_vp]),
    "vofp_last_error": (ctypes.c_char_p, [_vp]),
    "vofp_build_operator": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _P(_Bc), _P(_Phys)]),
    "vofp_rhs_from_face_velocity": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "vofp_project": (ctypes.c_int, [_vp] * 10 + [_P(ctypes.c_double)]),
    "vofp_exit_flux": (ctypes.c_int, [_vp] * 5 + [ctypes.c_double, _vp, ctypes.c_int, _vp, _P(ctypes.c_double)]),
    "vofp_vof_flux_correct": (ctypes.c_int, [_vp] * 11),
    "vofp_vof_advect": (ctypes.c_int, [_vp] * 9 + [ctypes.c_double, ctypes.c_int, _vp]),
    "vofp_rk2_step": (ctypes.c_int, [_vp] * 12 + [_P(_Bc), _P(_Phys), _P(_Opts), _vp, ctypes.c_int, _P(_Rk2Info)]),
    "vofp_apply": (ctypes.c_int, [_vp, _vp, _vp]),
    "vofp_residual": (ctypes.c_int, [_vp, _vp, _vp, _P(ctypes.c_double)]),
    "vofp_solve": (ctypes.c_int, [_vp, _vp, _vp, _P(_Opts), _P(_Info)]),
    "vofp_solve_host": (ctypes.c_int, [_vp] + [_vp] * 8 + [_P(_Bc), _P(_Phys), _P(_Opts), _vp, _P(_Info)]),
    "vofp_solve_host_batch": (ctypes.c_int, [_vp, ctypes.c_int, _P(_HostStep), _P(_Bc), _P(_Phys), _P(_Opts),
                                             _P(_Info)]),
    "vofp_merge_map": (ctypes.c_int, [_vp, _vp]),
    "vofp_get_stats": (ctypes.c_int, [_vp, _P(_Stats)]),
    "vofp_residual_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _P(ctypes.c_double)]),
    "vofp_launch_count": (ctypes.c_int, [_vp, _P(ctypes.c_longlong)]),
    "vofp_rbc_split_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int),
                                           _P(ctypes.c_int), _P(ctypes.c_int)]),
    "vofp_scaled_pair": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "vofp_measure_fma_peaks": (ctypes.c_int, [_vp, _P(ctypes.c_double), _P(ctypes.c_double)]),
    "vofp_nn_train_step_anorm": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_int,
                                                _P(ctypes.c_float)]),
    "vofp_nn_create": (ctypes.c_int, [_P(_vp), ctypes.c_ulonglong, _vp]),
    "vofp_nn_destroy": (None, [_vp]),
    "vofp_nn_last_error": (ctypes.c_char_p, [_vp]),
    "vofp_nn_param_count": (ctypes.c_int, [_vp, _P(ctypes.c_longlong)]),
    "vofp_nn_get_params": (ctypes.c_int, [_vp, _vp, ctypes.c_longlong, ctypes.c_int]),
    "vofp_nn_set_params": (ctypes.c_int, [_vp, _vp, ctypes.c_longlong]),
    "vofp_nn_bind": (ctypes.c_int, [_vp, _vp, _vp]),
    "vofp_nn_export_geometry": (ctypes.c_int, [_vp, _vp, _vp]),
    "vofp_nn_set_geometry": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "vofp_nn_forward": (ctypes.c_int, [_vp, _vp, _vp]),
    "vofp_nn_conv_apply": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _vp, _vp]),
    "vofp_nn_conv_wgrad": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                          _vp]),
    "vofp_nn_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_int, _P(ctypes.c_float)]),
    "vofp_time_iteration_kernels": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   _P(ctypes.c_float), _P(ctypes.c_float), _P(ctypes.c_float)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


def _check(ctx, status):
    if status != OK:
        msg = _lib.vofp_last_error(ctx)
        raise VofpError(status, msg.decode() if msg else "")


def _dev(t, n, name, dtype="float64"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype}" or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: need contiguous {dtype} with {n} elements, got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---- functions with the C names ------------------------------------------------------------

def vofp_version() -> str:
    return _lib.vofp_version().decode()


def vofp_rbc_split_plan(tiles_x, tiles_y, nz, slots):
    """(blocks, per, pad, gx, gy) of the colour-compact red-black iteration kernel's work split
    (host only)."""
    v = [ctypes.c_int(0) for _ in range(5)]
    _check(None, _lib.vofp_rbc_split_plan(int(tiles_x), int(tiles_y), int(nz), int(slots),
                                          *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def vofp_measure_fma_peaks(stream=None):
    """(FP64, FP32) fused multiply-add throughput of the current device in TFLOP/s."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(None, _lib.vofp_measure_fma_peaks(_stream_handle(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def vofp_create(dx, dy, dz, stream=None):
    dx, dy, dz = (np.ascontiguousarray(a, dtype=np.float64) for a in (dx, dy, dz))
    g = _Grid(len(dx), len(dy), len(dz), dx.ctypes.data_as(_P(ctypes.c_double)),
              dy.ctypes.data_as(_P(ctypes.c_double)), dz.ctypes.data_as(_P(ctypes.c_double)))
    h = _vp()
    st = _lib.vofp_create(ctypes.byref(h), ctypes.byref(g), _stream_handle(stream))
    if st != OK:
        raise VofpError(st, "vofp_create failed")
    return h


def vofp_destroy(ctx):
    _lib.vofp_destroy(ctx)


def vofp_last_error(ctx) -> str:
    return _lib.vofp_last_error(ctx).decode()


class Context:
    """One grid on one stream.  Arrays are torch CUDA float64 tensors in the layouts of vofp.h."""

    def __init__(self, dx, dy, dz, stream=None):
        self.nx, self.ny, self.nz = len(dx), len(dy), len(dz)
        self.n = self.nx * self.ny * self.nz
        self.nfx = (self.nx + 1) * self.ny * self.nz
        self.nfy = self.nx * (self.ny + 1) * self.nz
        self.nfz = self.nx * self.ny * (self.nz + 1)
        self.h = vofp_create(dx, dy, dz, stream)
        self._keep = []

    def close(self):
        if self.h:
            vofp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operator ------------------------------------------------------------------------------
    def _bc(self, kinds, neumann_flux):
        b = _Bc()
        self._keep = []
        for f in range(6):
            b.kind[f] = int(kinds[f])
            g = None if neumann_flux is None else neumann_flux[f]
            if g is None:
                b.neumann_flux[f] = None
            else:
                nb = (self.ny * self.nz, self.ny * self.nz, self.nx * self.nz, self.nx * self.nz,
                      self.nx * self.ny, self.nx * self.ny)[f]
                b.neumann_flux[f] = _dev(g, nb, f"neumann_flux[{f}]").value
                self._keep.append(g)
        return b

    def vofp_build_operator(self, F, ax, ay, az, vol_frac, bc, rho_liquid=1000.0, rho_gas=1.2,
                            merge_threshold=0.1, density_smoothing=0, dt=1.0, neumann_flux=None):
        b = self._bc(bc, neumann_flux)
        ph = _Phys(rho_liquid, rho_gas, merge_threshold, int(density_smoothing), dt)
        vf = None if vol_frac is None else _dev(vol_frac, self.n, "vol_frac")
        _check(self.h, _lib.vofp_build_operator(self.h, _dev(F, self.n, "F"), _dev(ax, self.nfx, "ax"),
                                                _dev(ay, self.nfy, "ay"), _dev(az, self.nfz, "az"),
                                                vf, ctypes.byref(b), ctypes.byref(ph)))

    def vofp_rhs_from_face_velocity(self, u, v, w, body_flux=None, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=u.device)
        bf = None if body_flux is None else _dev(body_flux, self.n, "body_flux")
        _check(self.h, _lib.vofp_rhs_from_face_velocity(self.h, _dev(u, self.nfx, "u"), _dev(v, self.nfy, "v"),
                                                        _dev(w, self.nfz, "w"), bf, _dev(out, self.n, "b")))
        return out

    def vofp_project(self, p, u, v, w, body_flux=None, out=None, want_div=True, want_max=True):
        """Projected face velocities (u, v, w), the group-folded divergence per cell (or None) and
        its max |.| (or None).  out = (u_out, v_out, w_out) may be the inputs themselves."""
        import torch
        if out is None:
            out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        uo, vo, wo = out
        div = torch.empty(self.n, dtype=torch.float64, device=p.device) if want_div else None
        m = ctypes.c_double(0.0)
        bf = None if body_flux is None else _dev(body_flux, self.n, "body_flux")
        _check(self.h, _lib.vofp_project(self.h, _dev(p, self.n, "p"), _dev(u, self.nfx, "u"),
                                         _dev(v, self.nfy, "v"), _dev(w, self.nfz, "w"), bf,
                                         _dev(uo, self.nfx, "u_out"), _dev(vo, self.nfy, "v_out"),
                                         _dev(wo, self.nfz, "w_out"),
                                         None if div is None else _dev(div, self.n, "div"),
                                         ctypes.byref(m) if want_max else None))
        return uo, vo, wo, div, (m.value if want_max else None)

    def vofp_exit_flux(self, u, v=None, w=None, u_c=0.0, R=None, balance=False, body_flux=None, out=None):
        """Exit flux of the radiation condition (Sec. 2.6, Eq. exit) from the x-face velocities u,
        installed as the +x face's prescribed flux; with balance, shifted over the open exit area so
        that the all-Neumann right-hand side sums to zero.  Returns (g on the (nz, ny) exit faces,
        the shift subtracted)."""
        import torch
        rows = self.nz * self.ny
        if out is None:
            out = torch.empty(rows, dtype=torch.float64, device=u.device)
        sh = ctypes.c_double(0.0)
        _check(self.h, _lib.vofp_exit_flux(self.h, _dev(u, self.nfx, "u"),
                                           None if v is None else _dev(v, self.nfy, "v"),
                                           None if w is None else _dev(w, self.nfz, "w"),
                                           None if body_flux is None else _dev(body_flux, self.n, "body_flux"),
                                           float(u_c), None if R is None else _dev(R, rows, "R"), int(bool(balance)),
                                           _dev(out, rows, "g"), ctypes.byref(sh)))
        return out, sh.value

    def vofp_vof_flux_correct(self, ax, ay, az, u, v, w):
        """Flux-error correction of Sec. 2.4: (ux^ on x faces, uy^ on y faces, wm^, wp^ per cell)."""
        import torch
        o = (torch.empty_like(u), torch.empty_like(v), torch.empty(self.n, dtype=torch.float64, device=u.device),
             torch.empty(self.n, dtype=torch.float64, device=u.device))
        _check(self.h, _lib.vofp_vof_flux_correct(self.h, _dev(ax, self.nfx, "ax"), _dev(ay, self.nfy, "ay"),
                                                  _dev(az, self.nfz, "az"), _dev(u, self.nfx, "u"),
                                                  _dev(v, self.nfy, "v"), _dev(w, self.nfz, "w"),
                                                  _dev(o[0], self.nfx, "ux_hat"), _dev(o[1], self.nfy, "uy_hat"),
                                                  _dev(o[2], self.n, "wm_hat"), _dev(o[3], self.n, "wp_hat")))
        return o

    def vofp_vof_advect(self, F, ax, ay, az, vol_frac, u, v, w, dt, order=0, out=None):
        """phi - VOF(u, phi, dt) of Sec. 2.4 (flux-error correction, three split stages)."""
        import torch
        if out is None:
            out = torch.empty_like(F)
        _check(self.h, _lib.vofp_vof_advect(self.h, _dev(F, self.n, "F"), _dev(ax, self.nfx, "ax"),
                                            _dev(ay, self.nfy, "ay"), _dev(az, self.nfz, "az"),
                                            _dev(vol_frac, self.n, "vol_frac"), _dev(u, self.nfx, "u"),
                                            _dev(v, self.nfy, "v"), _dev(w, self.nfz, "w"), float(dt), int(order),
                                            _dev(out, self.n, "F_out")))
        return out

    def vofp_rk2_step(self, F, ax, ay, az, vol_frac, u, v, w, bc, p, order=0, R=None, neumann_flux=None,
                      rho_liquid=1000.0, rho_gas=1.2, merge_threshold=0.1, density_smoothing=0, dt=1.0,
                      mode=MODE_MIXED, precond=PRECOND_RBSGS, rtol=1e-8, max_iter=100000, inner_rtol=0.0,
                      check_every=0, raise_on_error=True):
        """One RK2 step of Sec. 2.1 (two solves, two projections, two VOF steps); F, u, v, w and p
        are updated in place.  Returns the two solves' info dicts and the largest group divergence."""
        b = self._bc(bc, neumann_flux)
        ph = _Phys(float(rho_liquid), float(rho_gas), float(merge_threshold), int(density_smoothing), float(dt))
        o = _Opts(int(mode), int(precond), float(rtol), int(max_iter), float(inner_rtol), int(check_every), 0, 0,
                  None, 20, 0)
        info = _Rk2Info()
        Rs = (None, None, None) if R is None else (_dev(R[0], self.nfx, "Ru"), _dev(R[1], self.nfy, "Rv"),
                                                   _dev(R[2], self.nfz, "Rw"))
        st = _lib.vofp_rk2_step(self.h, _dev(F, self.n, "F"), _dev(ax, self.nfx, "ax"), _dev(ay, self.nfy, "ay"),
                                _dev(az, self.nfz, "az"), _dev(vol_frac, self.n, "vol_frac"), _dev(u, self.nfx, "u"),
                                _dev(v, self.nfy, "v"), _dev(w, self.nfz, "w"), *Rs, ctypes.byref(b),
                                ctypes.byref(ph), ctypes.byref(o), _dev(p, self.n, "p"), int(order),
                                ctypes.byref(info))
        if raise_on_error:
            _check(self.h, st)

        def d(i):
            return {"iterations": i.iterations, "outer_iterations": i.outer_iterations,
                    "rel_residual": i.rel_residual, "seconds": i.seconds, "status": i.status,
                    "status_name": STATUS_NAMES.get(i.status, str(i.status))}
        return d(info.solve1), d(info.solve2), info.max_div

    def vofp_apply(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=x.device)
        _check(self.h, _lib.vofp_apply(self.h, _dev(x, self.n, "x"), _dev(out, self.n, "y")))
        return out

    def vofp_residual(self, b, x) -> float:
        r = ctypes.c_double(0.0)
        _check(self.h, _lib.vofp_residual(self.h, _dev(b, self.n, "b"), _dev(x, self.n, "x"), ctypes.byref(r)))
        return r.value

    def vofp_residual_noalloc(self, b, x) -> float:
        """vofp_residual without any device allocation (fixed static scratch; see vofp.h)."""
        r = ctypes.c_double(0.0)
        _check(self.h, _lib.vofp_residual_noalloc(self.h, _dev(b, self.n, "b"), _dev(x, self.n, "x"),
                                                  ctypes.byref(r)))
        return r.value

    def vofp_solve(self, b, x=None, mode=MODE_FP64, rtol=1e-10, max_iter=100000, inner_rtol=0.0,
                   check_every=0, precond=PRECOND_JACOBI, raise_on_error=True, x0_zero=0, host_loop=0,
                   nn=None, stag_window=0, inner_restart=0, stag_ratio=0.0):
        import torch
        if x is None:
            x = torch.zeros(self.n, dtype=torch.float64, device=b.device)
            x0_zero = 1
        o = _Opts(int(mode), int(precond), float(rtol), int(max_iter), float(inner_rtol), int(check_every), x0_zero,
                  int(host_loop), nn.h if nn is not None else None, int(stag_window), int(inner_restart),
                  float(stag_ratio))
        info = _Info()
        st = _lib.vofp_solve(self.h, _dev(b, self.n, "b"), _dev(x, self.n, "x"), ctypes.byref(o), ctypes.byref(info))
        out = {"iterations": info.iterations, "outer_iterations": info.outer_iterations,
               "rel_residual": info.rel_residual, "seconds": info.seconds, "status": info.status,
               "status_name": STATUS_NAMES.get(info.status, str(info.status)),
               "nn_applications": info.nn_applications, "fell_back": info.fell_back}
        if st != OK and raise_on_error and st not in (ERR_NOT_CONVERGED,):
            _check(self.h, st)
        out["return_status"] = st
        return x, out

    @staticmethod
    def _host_ptr(a, n, name):
        """Address of a host float64 array of n values (numpy, or a torch CPU tensor, pinned or not)."""
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            if a.numel() != n or a.is_cuda:
                raise ValueError(name)
            return ctypes.c_void_p(a.data_ptr())
        # an ndarray itself (a converted copy would be freed before the call reads it)
        if not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.size != n or not a.flags.c_contiguous:
            raise ValueError(name)
        return ctypes.c_void_p(a.ctypes.data)

    def vofp_solve_host_batch(self, steps, bc, mode=MODE_FP64, rtol=1e-10, max_iter=100000, inner_rtol=0.0,
                              check_every=0, rho_liquid=1000.0, rho_gas=1.2, merge_threshold=0.1,
                              density_smoothing=0, dt=1.0, precond=PRECOND_JACOBI, inner_restart=0):
        """Independent host-buffer end-to-end solves in one call, the next step's uploads overlapping
        this step's solve.  steps: sequence of dicts with keys F, ax, ay, az, vol_frac (may be None),
        u, v, w and x_out (host float64 arrays; pinned torch tensors for the overlap).  Returns one
        info dict per step and the call's status."""
        hp = self._host_ptr
        if len(steps) < 1:
            raise ValueError("steps")
        arr = (_HostStep * len(steps))()
        for i, s in enumerate(steps):
            ptrs = (hp(s["F"], self.n, "F"), hp(s["ax"], self.nfx, "ax"), hp(s["ay"], self.nfy, "ay"),
                    hp(s["az"], self.nfz, "az"), hp(s.get("vol_frac"), self.n, "vol_frac"), hp(s["u"], self.nfx, "u"),
                    hp(s["v"], self.nfy, "v"), hp(s["w"], self.nfz, "w"), hp(s["x_out"], self.n, "x_out"))
            arr[i] = _HostStep(*[p.value if p is not None else None for p in ptrs])
        b = self._bc(bc, None)
        ph = _Phys(rho_liquid, rho_gas, merge_threshold, int(density_smoothing), dt)
        o = _Opts(int(mode), int(precond), float(rtol), int(max_iter), float(inner_rtol), int(check_every), 1, 0,
                  None, 0, int(inner_restart), 0.0)
        infos = (_Info * len(steps))()
        st = _lib.vofp_solve_host_batch(self.h, len(steps), arr, ctypes.byref(b), ctypes.byref(ph), ctypes.byref(o),
                                        infos)
        if st not in (OK, ERR_NOT_CONVERGED):
            _check(self.h, st)
        return [{"iterations": f.iterations, "outer_iterations": f.outer_iterations, "rel_residual": f.rel_residual,
                 "seconds": f.seconds, "status": f.status} for f in infos], st

    def vofp_solve_host(self, F, ax, ay, az, vol_frac, u, v, w, bc, x_out, mode=MODE_FP64, rtol=1e-10,
                        max_iter=100000, inner_rtol=0.0, check_every=0, rho_liquid=1000.0, rho_gas=1.2,
                        merge_threshold=0.1, density_smoothing=0, dt=1.0, precond=PRECOND_JACOBI, inner_restart=0):
        """Host-buffer end-to-end call: numpy (or pinned torch CPU) float64 arrays in, x_out out."""
        hp = self._host_ptr
        b = self._bc(bc, None)
        ph = _Phys(rho_liquid, rho_gas, merge_threshold, int(density_smoothing), dt)
        o = _Opts(int(mode), int(precond), float(rtol), int(max_iter), float(inner_rtol), int(check_every), 1, 0,
                  None, 0, int(inner_restart), 0.0)
        info = _Info()
        st = _lib.vofp_solve_host(self.h, hp(F, self.n, "F"), hp(ax, self.nfx, "ax"), hp(ay, self.nfy, "ay"),
                                  hp(az, self.nfz, "az"), hp(vol_frac, self.n, "vol_frac"), hp(u, self.nfx, "u"),
                                  hp(v, self.nfy, "v"), hp(w, self.nfz, "w"), ctypes.byref(b), ctypes.byref(ph),
                                  ctypes.byref(o), hp(x_out, self.n, "x_out"), ctypes.byref(info))
        if st not in (OK, ERR_NOT_CONVERGED):
            _check(self.h, st)
        return {"iterations": info.iterations, "outer_iterations": info.outer_iterations,
                "rel_residual": info.rel_residual, "seconds": info.seconds, "status": info.status}

    def vofp_scaled_pair(self, b, x):
        """(S b_hat, S^-1 x) as FP32 CUDA tensors: the network's input and target variables."""
        import torch
        r = torch.empty(self.n, dtype=torch.float32, device=b.device)
        xs = torch.empty(self.n, dtype=torch.float32, device=b.device)
        _check(self.h, _lib.vofp_scaled_pair(self.h, _dev(b, self.n, "b"), _dev(x, self.n, "x"),
                                             _dev(r, self.n, "r_scaled", "float32"),
                                             _dev(xs, self.n, "x_scaled", "float32")))
        return r, xs

    def vofp_merge_map(self):
        import torch
        out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        _check(self.h, _lib.vofp_merge_map(self.h, _dev(out, self.n, "master", "int32")))
        return out

    def vofp_get_stats(self):
        s = _Stats()
        _check(self.h, _lib.vofp_get_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def vofp_launch_count(self) -> int:
        n = ctypes.c_longlong(0)
        _check(self.h, _lib.vofp_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def vofp_time_iteration_kernels(self, precision=64, reps=20, precond=PRECOND_JACOBI):
        """Average device ms of one iteration's (stencil, update, fix-row + group) kernels; the
        third is 0 except for the FP32 red-black iteration on colour-compact vectors."""
        a, b, r = ctypes.c_float(0), ctypes.c_float(0), ctypes.c_float(0)
        _check(self.h, _lib.vofp_time_iteration_kernels(self.h, int(precision), int(precond), int(reps),
                                                        ctypes.byref(a), ctypes.byref(b), ctypes.byref(r)))
        return a.value, b.value, r.value


# (input, output) channels of the network's ten 3x3x3 convolutions, forward order
LAYER_CHANNELS = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]


class Network:
    """The learned preconditioner (vofp_nn_*): 3-level 3-D conv encoder-decoder, BF16 on tensor cores."""

    def __init__(self, seed=0, stream=None):
        self.h = _vp()
        st = _lib.vofp_nn_create(ctypes.byref(self.h), ctypes.c_ulonglong(seed), _stream_handle(stream))
        if st != OK:
            raise VofpError(st, "vofp_nn_create failed")
        n = ctypes.c_longlong(0)
        _lib.vofp_nn_param_count(self.h, ctypes.byref(n))
        self.nparams = n.value
        self.n = 0

    def _check(self, st):
        if st != OK:
            raise VofpError(st, _lib.vofp_nn_last_error(self.h).decode())

    def close(self):
        if self.h:
            _lib.vofp_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, grads=False):
        out = np.empty(self.nparams, dtype=np.float32)
        self._check(_lib.vofp_nn_get_params(self.h, ctypes.c_void_p(out.ctypes.data), self.nparams, int(grads)))
        return out

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        assert params.size == self.nparams
        self._check(_lib.vofp_nn_set_params(self.h, ctypes.c_void_p(params.ctypes.data), self.nparams))

    def bind(self, ctx, F):
        self._check(_lib.vofp_nn_bind(self.h, ctx.h, _dev(F, ctx.n, "F")))
        self.n = ctx.n
        self.shape = (ctx.nz, ctx.ny, ctx.nx)

    def export_geometry(self):
        import torch
        geo = torch.empty(self.n * 8, dtype=torch.int16, device="cuda")
        mask = torch.empty(self.n, dtype=torch.float32, device="cuda")
        self._check(_lib.vofp_nn_export_geometry(self.h, ctypes.c_void_p(geo.data_ptr()),
                                                 ctypes.c_void_p(mask.data_ptr())))
        return geo, mask

    def set_geometry(self, shape, geo, mask):
        nz, ny, nx = shape
        self.n = nx * ny * nz
        self.shape = shape
        self._check(_lib.vofp_nn_set_geometry(self.h, nx, ny, nz, ctypes.c_void_p(geo.data_ptr()),
                                              ctypes.c_void_p(mask.data_ptr())))

    def forward(self, r, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float32, device=r.device)
        self._check(_lib.vofp_nn_forward(self.h, _dev(r, self.n, "r", "float32"), _dev(out, self.n, "z", "float32")))
        return out

    def conv_apply(self, layer, x, shape, data_grad=False):
        """One convolution layer on a chunk-planar BF16 tensor x of shape (nz, ny, nx) voxels
        (vofp_nn_conv_apply); returns the chunk-planar BF16 output."""
        import torch
        nz, ny, nx = shape
        cin, cout = LAYER_CHANNELS[layer]
        cout_here = cin if data_grad else cout
        cin_here = cout if data_grad else cin
        V = nx * ny * nz
        if x.dtype != torch.bfloat16 or x.numel() != V * cin_here or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous chunk-planar CUDA bfloat16 tensor of the layer's input")
        out = torch.empty(V * cout_here, dtype=torch.bfloat16, device=x.device)
        self._check(_lib.vofp_nn_conv_apply(self.h, int(layer), int(bool(data_grad)), int(nx), int(ny), int(nz),
                                            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def conv_wgrad(self, layer, x, dy, shape):
        """Weight and bias gradients of one convolution layer from chunk-planar BF16 tensors x (its
        input) and dy (its output gradient) (vofp_nn_conv_wgrad); returns (gw [27][cout][cin], gb)."""
        import torch
        nz, ny, nx = shape
        cin, cout = LAYER_CHANNELS[layer]
        V = nx * ny * nz
        for t, c in ((x, cin), (dy, cout)):
            if t.dtype != torch.bfloat16 or t.numel() != V * c or not t.is_cuda or not t.is_contiguous():
                raise ValueError("x and dy must be contiguous chunk-planar CUDA bfloat16 tensors")
        gw = torch.empty(27 * cout * cin, dtype=torch.float32, device=x.device)
        gb = torch.empty(cout, dtype=torch.float32, device=x.device)
        self._check(_lib.vofp_nn_conv_wgrad(self.h, int(layer), int(nx), int(ny), int(nz),
                                            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(dy.data_ptr()),
                                            ctypes.c_void_p(gw.data_ptr()), ctypes.c_void_p(gb.data_ptr())))
        return gw.view(27, cout, cin), gb

    def train_step(self, r, target, lr=1e-3, update=True):
        loss = ctypes.c_float(0.0)
        self._check(_lib.vofp_nn_train_step(self.h, _dev(r, self.n, "r", "float32"),
                                            _dev(target, self.n, "target", "float32"), float(lr), int(update),
                                            ctypes.byref(loss)))
        return loss.value

    def train_step_anorm(self, ctx, r, e, lr=1e-3, update=True):
        """One step on the relative A-norm error of the output against the exact error e of the
        scaled residual r under ctx's operator (vofp_nn_train_step_anorm); returns the loss."""
        loss = ctypes.c_float(0.0)
        st = _lib.vofp_nn_train_step_anorm(self.h, ctx.h, _dev(r, self.n, "r", "float32"),
                                           _dev(e, self.n, "e", "float32"), float(lr), int(update),
                                           ctypes.byref(loss))
        if st != OK:
            raise VofpError(st, _lib.vofp_last_error(ctx.h).decode())
        return loss.value


def context_for(problem, stream=None, device="cuda"):
    """Create a Context for an inputs.Problem, upload its arrays and build the operator.
    Returns (ctx, device arrays dict)."""
    import torch
    ctx = Context(problem.dx, problem.dy, problem.dz, stream)
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(problem, k)).ravel()).to(device)
         for k in ("F", "vf", "ax", "ay", "az", "u", "v", "w")}
    ctx.vofp_build_operator(t["F"], t["ax"], t["ay"], t["az"], t["vf"], problem.bc,
                            problem.rho_liquid, problem.rho_gas, problem.merge_threshold,
                            problem.density_smoothing, problem.dt)
    return ctx, t
