"""ctypes binding of libsw (``include/sw.h``): the same entry points with the
same names, argument marshalling only.  Every step of the hot path runs in the
CUDA library; there is no Python or CPU fallback -- if the library is missing
or no GPU is present, the calls raise.

Low level: ``lib()`` returns the ``ctypes.CDLL`` with typed ``sw_*`` functions.
Convenience wrappers (:class:`Context`, :class:`Matrix`) marshal numpy host
arrays and torch device tensors to pointers.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

SW_OK, SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT, SW_ENONCONV, SW_ESTATE = range(7)
SW_FP64_PLAIN, SW_FP32_KAHAN = 0, 1
STATUS_NAMES = {0: "SW_OK", 1: "SW_EINVAL", 2: "SW_ENOMEM", 3: "SW_ECUDA", 4: "SW_ETIMEOUT", 5: "SW_ENONCONV",
                6: "SW_ESTATE"}


class SwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PotentialParams(ctypes.Structure):
    _fields_ = [("disc_M", ctypes.c_double), ("disc_a", ctypes.c_double), ("disc_b", ctypes.c_double),
                ("halo_M200", ctypes.c_double), ("halo_c", ctypes.c_double), ("H0", ctypes.c_double),
                ("bar_M", ctypes.c_double), ("bar_L", ctypes.c_double), ("bar_b", ctypes.c_double),
                ("bar_c", ctypes.c_double), ("test_kind", ctypes.c_int32), ("bar_kind", ctypes.c_int32),
                ("test_M", ctypes.c_double), ("test_a", ctypes.c_double)]


class PixelGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


class VBins(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("reserved", ctypes.c_int32), ("v0", ctypes.c_double),
                ("dv", ctypes.c_double)]


class DensityGrid(ctypes.Structure):
    _fields_ = [("nR", ctypes.c_int32), ("nphi", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("Rmax", ctypes.c_double), ("zmin", ctypes.c_double),
                ("zmax", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I64 = ctypes.POINTER(ctypes.c_int64)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_VP = ctypes.c_void_p
_lib = None

# (restype, argtypes) of every exported entry point, in include/sw.h order
SIGNATURES = {
    "sw_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, _VP]),
    "sw_destroy": (ctypes.c_int, [_VP]),
    "sw_last_error": (ctypes.c_char_p, [_VP]),
    "sw_set_potential": (ctypes.c_int, [_VP, ctypes.POINTER(PotentialParams)]),
    "sw_integrate_library": (ctypes.c_int, [_VP, _D, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int64, _D, _U8]),
    "sw_integrate_library_device": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_int64, _VP, _VP]),
    "sw_project": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(PixelGrid), ctypes.POINTER(VBins), ctypes.POINTER(DensityGrid), _D,
                                  ctypes.c_int, ctypes.POINTER(_VP)]),
    "sw_reduce_gh": (ctypes.c_int, [_VP, _VP, _D, ctypes.POINTER(_VP)]),
    "sw_bundle": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.POINTER(_VP)]),
    "sw_batch_create": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(_VP)]),
    "sw_batch_set_models": (ctypes.c_int, [_VP, _VP, _D, _D, ctypes.c_double, _D, _D]),
    "sw_batch_run": (ctypes.c_int, [_VP]),
    "sw_batch_matrix": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    "sw_batch_stats": (ctypes.c_int, [_VP, _D, _U8]),
    "sw_batch_info": (ctypes.c_int, [_VP, _VP, _D]),
    "sw_batch_destroy": (ctypes.c_int, [_VP]),
    "sw_mlp_param_count": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "sw_mlp_forward": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int64,
                                      ctypes.c_int, _VP]),
    "sw_mlp_loss_grad": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP,
                                        ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_double)]),
    "sw_mlp_adam": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "sw_project_stats": (ctypes.c_int, [_VP, _D, _U8]),
    "sw_solve_weights": (ctypes.c_int, [_VP, _VP, _D, _D, ctypes.c_double, _D, _D]),
    "sw_solve_weights_device": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP]),
    "sw_solve_info": (ctypes.c_int, [_VP, _D]),
    "sw_solve_bootstrap": (ctypes.c_int, [_VP, _VP, _D, _D, ctypes.c_double, ctypes.c_int64, _D, _D, _D, _D]),
    "sw_factor_preconditioner": (ctypes.c_int, [_VP, _F, ctypes.c_int64, ctypes.c_int, _F, _F, _I32]),
    "sw_matrix_shape": (ctypes.c_int, [_VP, _I64, _I64, _I64]),
    "sw_matrix_copy": (ctypes.c_int, [_VP, _D]),
    "sw_matrix_apply": (ctypes.c_int, [_VP, _D, _D]),
    "sw_matrix_apply_static": (ctypes.c_int, [_VP, _D, _D]),
    "sw_matrix_free": (ctypes.c_int, [_VP]),
    "sw_trajectory": (ctypes.c_int, [_VP, _D, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int64, _D]),
    "sw_potential_eval": (ctypes.c_int, [_VP, _D, ctypes.c_int64, _D, _D]),
    "sw_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sw_kernel_count": (ctypes.c_int, []),
    "sw_kernel_stats": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), _I64, _D]),
    "sw_reset_stats": (ctypes.c_int, [_VP]),
    "sw_kernel_work": (ctypes.c_int, [_VP, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    "sw_launch_count": (ctypes.c_int64, [_VP]),
    "sw_alloc_count": (ctypes.c_int64, [_VP]),
    "sw_set_option": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_double]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libsw.  Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libsw is not built ({path}); run __graft_entry__.build() first")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous, "expected a C-contiguous float64 array"
    return a.ctypes.data_as(_D)


def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous, "expected a C-contiguous float32 array"
    return a.ctypes.data_as(_F)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous, "expected a C-contiguous int32 array"
    return a.ctypes.data_as(_I32)


def _tp(t) -> int:
    """Device pointer of a CUDA torch tensor (contiguous)."""
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


def pixel_grid(g: dict) -> PixelGrid:
    nx, ny, pix = g["nx"], g["ny"], g["pix"]
    return PixelGrid(nx=nx, ny=ny, x0=-0.5 * nx * pix, y0=-0.5 * ny * pix, dx=pix, dy=pix)


def vbins(g: dict) -> VBins:
    nv, vmax = g.get("nv", 1), g.get("vmax", 400.0)
    return VBins(nv=nv, v0=-vmax, dv=2.0 * vmax / nv)


def density_grid(g: dict) -> DensityGrid:
    return DensityGrid(nR=g["nR"], nphi=g["nphi"], nz=g["nz"], Rmax=g.get("Rmax", 10.0), zmin=g.get("zmin", -3.0),
                       zmax=g.get("zmax", 3.0))


def potential_params(p: dict) -> PotentialParams:
    return PotentialParams(disc_M=p.get("disc_M", 0.0), disc_a=p.get("disc_a", 1.0), disc_b=p.get("disc_b", 1.0),
                           halo_M200=p.get("halo_M200", 0.0), halo_c=p.get("halo_c", 10.0), H0=p.get("H0", 70.0),
                           bar_M=p.get("bar_M", 0.0), bar_L=p.get("bar_L", 1.0), bar_b=p.get("bar_b", 1.0),
                           bar_c=p.get("bar_c", 1.0), test_kind=int(p.get("test_kind", 0)),
                           bar_kind=int(p.get("bar_kind", 0)), test_M=p.get("test_M", 0.0),
                           test_a=p.get("test_a", 1.0))


class Matrix:
    """Device-resident orbit matrix returned by :meth:`Context.project`."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx, self.handle = ctx, handle
        M, N = ctypes.c_int64(), ctypes.c_int64()
        b = (ctypes.c_int64 * 3)()
        lib().sw_matrix_shape(handle, ctypes.byref(M), ctypes.byref(N), b)
        self.M, self.N = M.value, N.value
        self.blocks = (b[0], b[1], b[2])

    def copy(self) -> np.ndarray:
        """U as float64, orbit-major (N, M)."""
        out = np.empty((self.N, self.M))
        self.ctx._check(lib().sw_matrix_copy(self.handle, _dp(out)))
        return out

    def apply(self, w: np.ndarray) -> np.ndarray:
        """U w (FP64 accumulation on the device)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        y = np.empty(self.M)
        self.ctx._check(lib().sw_matrix_apply(self.handle, _dp(w), _dp(y)))
        return y

    def apply_static(self, w: np.ndarray) -> np.ndarray:
        """U w through the entry point that allocates no device memory (static scratch)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        y = np.empty(self.M)
        self.ctx._check(lib().sw_matrix_apply_static(self.handle, _dp(w), _dp(y)))
        return y

    def free(self) -> None:
        if self.handle and not getattr(self, "borrowed", False):
            lib().sw_matrix_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Many trial models built in one persistent launch (see sw_batch_* in include/sw.h)."""

    def __init__(self, ctx: "Context", n_orb, nsteps: int, grid: dict):
        self.ctx = ctx
        self.n_orb = np.ascontiguousarray(n_orb, dtype=np.int64)
        self.grid = dict(grid)
        self._pg, self._vb, self._dg = pixel_grid(grid), vbins(grid), density_grid(grid)
        gh = int(bool(grid.get("gh")))
        h = _VP()
        ctx._check(lib().sw_batch_create(ctx.handle, len(self.n_orb), self.n_orb.ctypes.data_as(_VP), int(nsteps),
                                         ctypes.byref(self._pg), None if gh else ctypes.byref(self._vb),
                                         ctypes.byref(self._dg), gh, int(grid.get("mirror4", 1)), ctypes.byref(h)))
        self.handle = h.value

    def set_models(self, pots: list, omega_p, angles, dt: float, ics: np.ndarray, gh_v0s: Optional[np.ndarray] = None):
        arr = (PotentialParams * len(pots))(*[potential_params(p) for p in pots])
        om = np.ascontiguousarray(omega_p, dtype=np.float64)
        an = np.ascontiguousarray(angles, dtype=np.float64).reshape(-1)
        ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1)
        gh = None
        if gh_v0s is not None:
            gh_v0s = np.ascontiguousarray(gh_v0s, dtype=np.float64).reshape(-1)
            gh = _dp(gh_v0s)
        self.ctx._check(lib().sw_batch_set_models(self.handle, arr, _dp(om), _dp(an), dt, _dp(ics), gh))

    def run(self) -> None:
        self.ctx._check(lib().sw_batch_run(self.handle))

    def matrix(self, k: int) -> Matrix:
        out = _VP()
        self.ctx._check(lib().sw_batch_matrix(self.handle, int(k), ctypes.byref(out)))
        m = Matrix(self.ctx, out.value)
        m.borrowed = True
        return m

    def stats(self):
        n = int(self.n_orb.sum())
        drift = np.empty(n); status = np.empty(n, dtype=np.uint8)
        self.ctx._check(lib().sw_batch_stats(self.handle, _dp(drift), status.ctypes.data_as(_U8)))
        return drift, status

    def info(self) -> dict:
        i4 = (ctypes.c_int64 * 4)()
        t = np.empty(12)
        self.ctx._check(lib().sw_batch_info(self.handle, i4, _dp(t)))
        return {"threads": i4[0], "ctas": i4[1], "autotuned": bool(i4[2]), "graph": bool(i4[3]),
                "probe_ms": t.tolist()}

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().sw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One libsw context (one device, one precision, one stream)."""

    def __init__(self, device: int = 0, precision: str = "fp32", stream: Optional[int] = None):
        prec = {"fp32": SW_FP32_KAHAN, "fp64": SW_FP64_PLAIN}[precision]
        h = _VP()
        st = lib().sw_create(ctypes.byref(h), device, prec, stream)
        if st != SW_OK:
            raise SwError(st, "sw_create failed (no CUDA device?)")
        self.handle = h.value
        self.precision = precision
        self.device = device
        self.last_status = SW_OK   # status of the last solve_weights call

    def _check(self, st: int) -> int:
        if st not in (SW_OK,):
            raise SwError(st, lib().sw_last_error(self.handle).decode())
        return st

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().sw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: str, value: float) -> None:
        self._check(lib().sw_set_option(self.handle, key.encode(), float(value)))

    def set_potential(self, p: dict) -> None:
        pp = potential_params(p)
        self._check(lib().sw_set_potential(self.handle, ctypes.byref(pp)))

    def integrate_library(self, ics: np.ndarray, omega_p: float, dt: float, nsteps: int, want_drift: bool = False):
        ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
        n = len(ics)
        if want_drift:
            drift = np.empty(n); status = np.empty(n, dtype=np.uint8)
            self._check(lib().sw_integrate_library(self.handle, _dp(ics), n, omega_p, dt, nsteps, _dp(drift),
                                                   status.ctypes.data_as(_U8)))
            return drift, status
        self._check(lib().sw_integrate_library(self.handle, _dp(ics), n, omega_p, dt, nsteps, None, None))
        return None

    def integrate_library_device(self, ics_t, omega_p: float, dt: float, nsteps: int, drift_t=None, status_t=None):
        n = ics_t.numel() // 6
        self._check(lib().sw_integrate_library_device(self.handle, _tp(ics_t), n, omega_p, dt, nsteps,
                                                      _tp(drift_t) if drift_t is not None else None,
                                                      _tp(status_t) if status_t is not None else None))

    def project(self, grid: dict, gh_v0s: Optional[np.ndarray] = None) -> Matrix:
        pg, vb, dg = pixel_grid(grid), vbins(grid), density_grid(grid)
        out = _VP()
        gh = None
        if grid.get("gh"):
            assert gh_v0s is not None, "GH rows need the per-pixel reference (v0, s)"
            gh_v0s = np.ascontiguousarray(gh_v0s, dtype=np.float64)
            gh = _dp(gh_v0s)
        self._check(lib().sw_project(self.handle, grid["incl"], grid.get("pa", 0.0), grid.get("bar_angle", 0.0),
                                     ctypes.byref(pg), ctypes.byref(vb), ctypes.byref(dg), gh,
                                     int(grid.get("mirror4", 1)), ctypes.byref(out)))
        return Matrix(self, out.value)

    def reduce_gh(self, U: Matrix, gh_v0s: np.ndarray) -> Matrix:
        gh_v0s = np.ascontiguousarray(gh_v0s, dtype=np.float64)
        out = _VP()
        self._check(lib().sw_reduce_gh(self.handle, U.handle, _dp(gh_v0s), ctypes.byref(out)))
        return Matrix(self, out.value)

    def bundle(self, U: Matrix, n: int) -> Matrix:
        """Mean of each run of n consecutive columns (orbit bundles of n dithers)."""
        out = _VP()
        self._check(lib().sw_bundle(self.handle, U.handle, int(n), ctypes.byref(out)))
        return Matrix(self, out.value)

    # ---- learned chi^2 emulator (device pointers, e.g. torch tensors' data_ptr())
    def mlp_forward(self, shape, params_ptr: int, x_ptr: int, batch: int, out_ptr: int, bf16: bool = False):
        self._check(lib().sw_mlp_forward(self.handle, *shape, params_ptr, x_ptr, int(batch), int(bool(bf16)),
                                         out_ptr))

    def mlp_loss_grad(self, shape, params_ptr: int, x_ptr: int, t_ptr: int, batch: int, grad_ptr: int) -> float:
        loss = ctypes.c_double()
        self._check(lib().sw_mlp_loss_grad(self.handle, *shape, params_ptr, x_ptr, t_ptr, int(batch), grad_ptr,
                                           ctypes.byref(loss)))
        return loss.value

    def mlp_adam(self, n: int, params_ptr: int, grad_ptr: int, m_ptr: int, v_ptr: int, step: int, lr: float,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._check(lib().sw_mlp_adam(self.handle, int(n), params_ptr, grad_ptr, m_ptr, v_ptr, int(step), lr,
                                      beta1, beta2, eps))

    def project_stats(self, n: int):
        drift = np.empty(n); status = np.empty(n, dtype=np.uint8)
        self._check(lib().sw_project_stats(self.handle, _dp(drift), status.ctypes.data_as(_U8)))
        return drift, status

    def solve_weights(self, U: Matrix, data: np.ndarray, errors: np.ndarray, lam: float, allow_nonconv=False):
        data = np.ascontiguousarray(data, dtype=np.float64)
        errors = np.ascontiguousarray(errors, dtype=np.float64)
        w = np.empty(U.N); chi2 = np.empty(3)
        st = lib().sw_solve_weights(self.handle, U.handle, _dp(data), _dp(errors), lam, _dp(w), _dp(chi2))
        self.last_status = st
        if not (allow_nonconv and st == SW_ENONCONV):
            self._check(st)
        return w, chi2

    def solve_weights_device(self, U: Matrix, data_t, errors_t, lam: float, w_t, chi2_t) -> int:
        return lib().sw_solve_weights_device(self.handle, U.handle, _tp(data_t), _tp(errors_t), lam, _tp(w_t),
                                             _tp(chi2_t))

    def solve_bootstrap(self, U: Matrix, data: np.ndarray, errors: np.ndarray, lam: float, xi: np.ndarray,
                        want_weights: bool = False, allow_nonconv: bool = False):
        """(weights (B, N) or None, chi2_b (B,), chi2_model) of sw_solve_bootstrap; xi is (B, M)."""
        data = np.ascontiguousarray(data, dtype=np.float64)
        errors = np.ascontiguousarray(errors, dtype=np.float64)
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, U.M)
        B = len(xi)
        w = np.empty((B, U.N)) if want_weights else None
        chi_b = np.empty(B)
        chi_m = np.empty(1)
        st = lib().sw_solve_bootstrap(self.handle, U.handle, _dp(data), _dp(errors), lam, B, _dp(xi),
                                      _dp(w) if w is not None else None, _dp(chi_b), _dp(chi_m))
        if not (st == SW_OK or (allow_nonconv and st == SW_ENONCONV)):
            self._check(st)
        return w, chi_b, float(chi_m[0])

    def solve_info(self) -> dict:
        out = np.zeros(8)
        self._check(lib().sw_solve_info(self.handle, _dp(out)))
        return {"admm_iterations": int(out[0]), "refine_rounds": int(out[1]), "kkt_rel": float(out[2]),
                "constraint_space": bool(out[3]), "polish_solves": int(out[4]), "kkt_met": bool(out[5]),
                "ws_rounds": int(out[6]), "ws_size": int(out[7])}

    def trajectory(self, ics: np.ndarray, omega_p: float, dt: float, nsteps: int) -> np.ndarray:
        ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
        out = np.empty((len(ics), nsteps + 1, 6))
        self._check(lib().sw_trajectory(self.handle, _dp(ics), len(ics), omega_p, dt, nsteps, _dp(out)))
        return out

    def potential_eval(self, xyz: np.ndarray):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        phi = np.empty(len(xyz)); acc = np.empty((len(xyz), 3))
        self._check(lib().sw_potential_eval(self.handle, _dp(xyz), len(xyz), _dp(phi), _dp(acc)))
        return phi, acc

    # ---- profiling
    def set_profiling(self, on: bool) -> None:
        self._check(lib().sw_set_profiling(self.handle, int(bool(on))))

    def reset_stats(self) -> None:
        self._check(lib().sw_reset_stats(self.handle))

    def kernel_stats(self) -> dict:
        out = {}
        for k in range(lib().sw_kernel_count()):
            name = ctypes.c_char_p(); n = ctypes.c_int64(); ms = ctypes.c_double()
            self._check(lib().sw_kernel_stats(self.handle, k, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)))
            if n.value:
                work, kind = ctypes.c_double(), ctypes.c_int()
                self._check(lib().sw_kernel_work(self.handle, k, ctypes.byref(work), ctypes.byref(kind)))
                out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "work": work.value,
                                            "kind": ["none", "flop_simt", "flop_tensor", "bytes",
                                                     "orbit_steps"][kind.value]}
        return out

    def launch_count(self) -> int:
        return lib().sw_launch_count(self.handle)

    def factor_preconditioner(self, gram: np.ndarray, mode: int = 0):
        """(L, X = L^-1, info) of sw_factor_preconditioner for a K x K FP32 matrix (lower triangle read)."""
        G = np.ascontiguousarray(gram, dtype=np.float32)
        K = G.shape[0]
        assert G.shape == (K, K)
        L = np.empty((K, K), np.float32)
        X = np.empty((K, K), np.float32)
        info = np.zeros(1, np.int32)
        self._check(lib().sw_factor_preconditioner(self.handle, _fp(G), K, mode, _fp(L), _fp(X), _ip(info)))
        return L, X, int(info[0])

    def alloc_count(self) -> int:
        return lib().sw_alloc_count(self.handle)
