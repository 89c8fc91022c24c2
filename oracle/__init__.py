"""FP64 CPU oracle for the Schwarzschild orbit-library hot path (arxiv 2607.00117).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path and never imports the product package.

Contents
--------
* ctypes wrappers over ``oracle.c`` (potentials, KDK integrator, Jacobi drift,
  mirrors, Euler projection, binning, Gauss-Hermite rows) -- Sec. 2.1-2.2.
* the weight problem of Sec. 2.3 in plain numpy FP64: whitening, the exact
  minimiser by Lawson-Hanson (on the stacked least-squares system and on its
  normal equations), brute-force support enumeration, the KKT certificate, the
  paper's ADMM, and chi^2 (Sec. 2.4).
* the chi^2 emulator MLP (12 -> 256 -> 256 -> 256 -> 1, SiLU) forward pass,
  hand-written backward pass and Adam step in FP64.
"""
from __future__ import annotations

import ctypes
import math
import itertools
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

G = 4.300917e-6  # kpc (km/s)^2 / Msun


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain IEEE double, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", src, "-o", _LIB_PATH + ".tmp", "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Pot(ctypes.Structure):
    _fields_ = [("disc_M", ctypes.c_double), ("disc_a", ctypes.c_double), ("disc_b", ctypes.c_double),
                ("halo_Mdm", ctypes.c_double), ("halo_rs", ctypes.c_double),
                ("bar_M", ctypes.c_double), ("bar_L", ctypes.c_double), ("bar_a", ctypes.c_double),
                ("bar_b", ctypes.c_double), ("test_kind", ctypes.c_int32), ("bar_kind", ctypes.c_int32),
                ("test_M", ctypes.c_double), ("test_a", ctypes.c_double)]


class Obs(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("nv", ctypes.c_int32), ("pad0", ctypes.c_int32), ("v0", ctypes.c_double), ("dv", ctypes.c_double),
                ("nR", ctypes.c_int32), ("nphi", ctypes.c_int32), ("nz", ctypes.c_int32), ("pad1", ctypes.c_int32),
                ("Rmax", ctypes.c_double), ("zmin", ctypes.c_double), ("zmax", ctypes.c_double),
                ("gh", ctypes.c_int32), ("mirror4", ctypes.c_int32)]


class BS3Opts(ctypes.Structure):
    """Adaptive Bogacki-Shampine 3(2) controls (Sec. 2.2.2): relative tolerance,
    first trial step, step-size controller, fixed-step switch, rejection cap."""
    _fields_ = [("rtol", ctypes.c_double), ("h0", ctypes.c_double), ("safety", ctypes.c_double),
                ("fac_min", ctypes.c_double), ("fac_max", ctypes.c_double), ("fixed", ctypes.c_int32),
                ("max_reject", ctypes.c_int32)]


DISC, HALO, BAR, TEST = 1, 2, 4, 8
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P, O = ctypes.POINTER(Pot), ctypes.POINTER(Obs)
        i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "orc_nfw_from_m200": (None, [dbl, dbl, dbl, _D, _D]),
            "orc_nfw_enclosed": (dbl, [dbl, dbl, dbl]),
            "orc_potential_eval": (None, [P, i32, i64, _D, _D, _D]),
            "orc_density_eval": (None, [P, i32, i64, _D, _D, i32]),
            "orc_jacobi": (dbl, [P, dbl, dbl, _D]),
            "orc_trajectory": (None, [P, dbl, dbl, i64, _D, _D]),
            "orc_drift": (None, [P, dbl, dbl, i64, i64, _D, _D]),
            "orc_euler_matrix": (None, [dbl, dbl, dbl, _D]),
            "orc_n_rows": (i64, [O]),
            "orc_build_matrix": (None, [P, dbl, dbl, i64, i64, _D, O, _D, _D, _D, _I32]),
            "orc_apply_matrix": (None, [P, dbl, dbl, i64, i64, _D, O, _D, _D, _D]),
            "orc_pixel_moments": (None, [P, dbl, dbl, i64, i64, _D, O, _D, _D]),
            "orc_gh_weights": (None, [dbl, _D]),
            "orc_bs3_trajectory": (i64, [P, dbl, ctypes.POINTER(BS3Opts), i64, _D, _D, _D]),
            "orc_build_matrix_bs3": (None, [P, dbl, ctypes.POINTER(BS3Opts), i64, i64, _D, O, _D, _D, _D, _I32]),
            "orc_bs3_single_step": (None, [P, dbl, dbl, _D, _D, _D]),
            "orc_jacobi_rot": (dbl, [P, dbl, _D]),
            "orc_max_threads": (i32, []),
            "orc_set_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


# ---------------------------------------------------------------------------
# Potential setup (Sec. 3.2.1-3.2.2, Eq. Rn_to_In)
# ---------------------------------------------------------------------------
def nfw_from_m200(M200: float, c: float, H0: float = 70.0):
    """(M200, c, H0) -> (M_DM, R_s), Sec. 3.2.1 with Delta_crit = 200."""
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_nfw_from_m200(M200, c, H0, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def nfw_enclosed(Mdm: float, rs: float, R: float) -> float:
    return lib().orc_nfw_enclosed(Mdm, rs, R)


def make_pot(p: dict) -> Pot:
    """Potential parameters -> oracle struct.  Keys as in the C-ABI's
    sw_potential_params: disc_M/a/b, halo_M200/c, H0, bar_M/L/b/c, test_kind/M/a.
    The bar's (L, b, c) are the needle half-length and the parent MN's radial
    scale and height (Eq. Rn_to_In with Z = a + zeta)."""
    Mdm, rs = (0.0, 1.0)
    if p.get("halo_M200", 0.0) > 0.0:
        Mdm, rs = nfw_from_m200(p["halo_M200"], p["halo_c"], p.get("H0", 70.0))
    return Pot(disc_M=p.get("disc_M", 0.0), disc_a=p.get("disc_a", 1.0), disc_b=p.get("disc_b", 1.0),
               halo_Mdm=Mdm, halo_rs=rs,
               bar_M=p.get("bar_M", 0.0), bar_L=p.get("bar_L", 1.0), bar_a=p.get("bar_b", 1.0),
               bar_b=p.get("bar_c", 1.0), test_kind=int(p.get("test_kind", 0)), bar_kind=int(p.get("bar_kind", 0)),
               test_M=p.get("test_M", 0.0), test_a=p.get("test_a", 1.0))


def potential(pot: Pot, xyz: np.ndarray, mask: int = DISC | HALO | BAR | TEST):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    phi = np.zeros(len(xyz)); acc = np.zeros((len(xyz), 3))
    lib().orc_potential_eval(ctypes.byref(pot), mask, len(xyz), _dp(xyz), _dp(phi), _dp(acc))
    return phi, acc


def density(pot: Pot, xyz: np.ndarray, mask: int = DISC | HALO | BAR | TEST, bar_nodes: int = 64):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    rho = np.zeros(len(xyz))
    lib().orc_density_eval(ctypes.byref(pot), mask, len(xyz), _dp(xyz), _dp(rho), bar_nodes)
    return rho


# ---------------------------------------------------------------------------
# The paper's bar (Sec. 2.1.2, App. A): Dehnen & Aly (2023) T3 and V4 parent pairs
# convolved with a needle along x, R^-n -> I_n (Eq. Rn_to_In)
# ---------------------------------------------------------------------------
_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def needle_In(x, y, Z, n: int, L: float, eta: float) -> np.ndarray:
    """I_n(x, y, Z) = int_{x-L}^{x+L} f(x - x') [x'^2 + y^2 + Z^2]^(-n/2) dx' with
    f(u) = [1 + eta (1 - 2|u|/L)] / (2L) (Eq. Rn_to_In), by 48-point Gauss-Legendre
    quadrature on the pieces between x - L, 0, x and x + L (the integrand's peak at
    x' = 0 and the needle's kink at x' = x)."""
    x, y, Z = (np.asarray(v, dtype=np.float64) for v in np.broadcast_arrays(x, y, Z))
    q2 = y * y + Z * Z
    lo, hi = x - L, x + L
    c1 = np.clip(0.0, lo, x)
    c2 = np.clip(0.0, x, hi)
    out = np.zeros_like(x)
    for a, b in ((lo, c1), (c1, x), (x, c2), (c2, hi)):
        half = 0.5 * (b - a)
        xp = (0.5 * (a + b))[..., None] + half[..., None] * _GL_X
        u = np.abs(x[..., None] - xp)
        f = (1.0 + eta * (1.0 - 2.0 * u / L)) / (2.0 * L)
        out += half * (f * (xp * xp + q2[..., None]) ** (-0.5 * n) * _GL_W).sum(-1)
    return out


def needle_In_closed(x, y, Z, n: int, L: float, eta: float) -> np.ndarray:
    """The same I_n (odd n) in closed form, as a kernel would evaluate it: with
    S(t) = sqrt(t^2 + q^2), q^2 = y^2 + Z^2, the antiderivatives
      J_1 = asinh(t/q),  J_{n+2} = [t S^-n + (n - 1) J_n] / (n q^2),
      K_n = int t S^-n dt = S^(2-n) / (2 - n)   (K_1 = S),
    and f(u) = [(1 + eta) - 2 eta |u| / L] / (2L) split at t = x."""
    x, y, Z = (np.asarray(v, dtype=np.float64) for v in np.broadcast_arrays(x, y, Z))
    q2 = y * y + Z * Z
    q = np.sqrt(q2)

    def J(t):
        S = np.sqrt(t * t + q2)
        j = np.arcsinh(t / q)
        for m in range(1, n, 2):
            j = (t * S ** (-m) + (m - 1) * j) / (m * q2)
        return j

    def K(t):
        S = np.sqrt(t * t + q2)
        return S ** (2 - n) / (2 - n)

    lo, hi = x - L, x + L
    Jlo, Jx, Jhi = J(lo), J(x), J(hi)
    Klo, Kx, Khi = K(lo), K(x), K(hi)
    flat = (Jhi - Jlo) / (2 * L)
    left = x * (Jx - Jlo) - (Kx - Klo)          # int_{x-L}^{x} (x - t) S^-n dt
    right = (Khi - Kx) - x * (Jhi - Jx)         # int_{x}^{x+L} (t - x) S^-n dt
    return (1 + eta) * flat - eta / (L * L) * (left + right)


def _da_terms(family: str, a: float, b: float, z):
    """Coefficients c_n(z) of the parent pair, Phi = -G M sum_n c_n R^-n and
    rho = M sum_n d_n R^-n (App. A), as functions of Z = a + zeta, zeta = sqrt(z^2 + b^2)."""
    zeta = np.sqrt(np.asarray(z, dtype=np.float64) ** 2 + b * b)
    Z = a + zeta
    if family == "T3":
        phi = {1: np.ones_like(Z), 3: a * (Z - a / 3.0), 5: a * a * Z * Z}
        k = b * b / (4.0 * math.pi)
        rho = {5: 3.0 * k * np.ones_like(Z),
               7: k * 5.0 * a * Z * Z * (3.0 * zeta ** 2 - 2.0 * a * zeta + a * a) / zeta ** 3,
               9: k * 35.0 * a * a * Z ** 4 / zeta ** 2}
    elif family == "V4":
        phi = {1: np.ones_like(Z), 3: a * (Z - 2.0 * a / 5.0) + b * b / 2.0,
               5: 3.0 * a * (a * Z * (2.0 * Z - a) / 5.0 + b * b / 2.0 * (Z - a / 5.0)),
               7: a * a * Z * Z * (a * Z + 3.0 * b * b), 9: 7.0 * a ** 3 * b * b * Z ** 4 / (2.0 * zeta)}
        k = 3.0 * b ** 4 / (8.0 * math.pi)
        rho = {7: 5.0 * k * np.ones_like(Z),
               9: k * 7.0 * a * Z * Z * (5 * zeta ** 4 - 4 * a * zeta ** 3 + 3 * a * a * zeta ** 2 - 2 * a ** 3 * zeta
                                         + a ** 4) / zeta ** 5,
               11: k * 63.0 * a * a * Z ** 4 * (2 * zeta ** 2 - 2 * a * zeta + a * a) / zeta ** 4,
               13: k * 231.0 * a ** 3 * Z ** 6 / zeta ** 3}
    else:
        raise ValueError(family)
    return Z, phi, rho


def dehnen_aly(family: str, M: float, a: float, b: float, L: float, eta: float, xyz: np.ndarray):
    """Potential and density of a Dehnen-Aly barred component (family 'T3' or 'V4';
    mass M, parent scales a, b, needle half-length L, slope eta) at bar-frame points
    (n, 3).  L = 0 gives the axisymmetric parent."""
    xyz = np.atleast_2d(np.asarray(xyz, dtype=np.float64))
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    Z, cphi, crho = _da_terms(family, a, b, z)

    def In(n):
        if L == 0.0:
            return (x * x + y * y + Z * Z) ** (-0.5 * n)
        return needle_In(x, y, Z, n, L, eta)

    phi = -G * M * sum(c * In(n) for n, c in cphi.items())
    rho = M * sum(c * In(n) for n, c in crho.items())
    return phi, rho


def paper_bar(M_b: float, L_b: float, b_d: float, xyz: np.ndarray, split_mass: float = 0.5):
    """The paper's composite bar (Sec. 2.1.2): a T3 long bar (eta = 1, a = L_b/5, b = b_d,
    L = L_b) plus a V4 boxy/peanut bulge (eta = 0, a = b = 0.5 kpc, L = 0.1 kpc) with tied
    masses; split_mass is the T3 share of M_b (0.5: equal masses summing to M_b)."""
    p1, r1 = dehnen_aly("T3", split_mass * M_b, L_b / 5.0, b_d, L_b, 1.0, xyz)
    p2, r2 = dehnen_aly("V4", (1.0 - split_mass) * M_b, 0.5, 0.5, 0.1, 0.0, xyz)
    return p1 + p2, r1 + r2


# ---------------------------------------------------------------------------
# Integration (Sec. 2.2.2)
# ---------------------------------------------------------------------------
def trajectory(pot: Pot, omega: float, dt: float, nsteps: int, ic) -> np.ndarray:
    ic = np.ascontiguousarray(ic, dtype=np.float64).reshape(6)
    out = np.zeros((nsteps + 1, 6))
    lib().orc_trajectory(ctypes.byref(pot), omega, dt, nsteps, _dp(ic), _dp(out))
    return out


def jacobi(pot: Pot, omega: float, t: float, state) -> float:
    s = np.ascontiguousarray(state, dtype=np.float64).reshape(6)
    return lib().orc_jacobi(ctypes.byref(pot), omega, t, _dp(s))


def drift(pot: Pot, omega: float, dt: float, nsteps: int, ics: np.ndarray) -> np.ndarray:
    ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
    out = np.zeros(len(ics))
    lib().orc_drift(ctypes.byref(pot), omega, dt, nsteps, len(ics), _dp(ics), _dp(out))
    return out


# ---------------------------------------------------------------------------
# The paper's adaptive integrator (Sec. 2.2.2): Bogacki-Shampine 3(2) in the
# bar frame, a fixed number of accepted steps, samples weighted by their step
# ---------------------------------------------------------------------------
def bs3_opts(rtol: float = 1e-4, h0: float = 5.11356e-4, safety: float = 0.9, fac_min: float = 0.2,
             fac_max: float = 5.0, fixed: bool = False, max_reject: int = 50) -> BS3Opts:
    """Controller readings (the paper gives only rtol = 1e-4 and the step count):
    error ratio max(|e_x| / (rtol max|x|), |e_v| / (rtol max|v|)) over the step,
    next step h (safety r^(-1/3)) clipped to [fac_min, fac_max] h, first trial
    step 0.5 Myr."""
    return BS3Opts(rtol=rtol, h0=h0, safety=safety, fac_min=fac_min, fac_max=fac_max, fixed=int(fixed),
                   max_reject=max_reject)


def bs3_trajectory(pot: Pot, omega: float, opts: BS3Opts, nsteps: int, ic):
    """(times (nsteps+1,), rotating-frame states (nsteps+1, 6), rejected trial
    steps; -1 when the orbit was abandoned) from an inertial initial condition."""
    ic = np.ascontiguousarray(ic, dtype=np.float64).reshape(6)
    ts = np.zeros(nsteps + 1)
    ys = np.zeros((nsteps + 1, 6))
    rej = lib().orc_bs3_trajectory(ctypes.byref(pot), omega, ctypes.byref(opts), nsteps, _dp(ic), _dp(ts), _dp(ys))
    return ts, ys, int(rej)


def rotating_to_inertial(omega: float, t: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """Rotating-frame states at times t -> inertial (x, v): rotate the position and
    v_rot + Omega z^ x x by R_z(Omega t)."""
    t = np.asarray(t, dtype=np.float64)
    c, s = np.cos(omega * t), np.sin(omega * t)
    x, y, z = ys[:, 0], ys[:, 1], ys[:, 2]
    vx, vy, vz = ys[:, 3] - omega * y, ys[:, 4] + omega * x, ys[:, 5]
    return np.stack([c * x - s * y, s * x + c * y, z, c * vx - s * vy, s * vx + c * vy, vz], 1)


def bs3_single_step(pot: Pot, omega: float, h: float, y):
    """One step from a rotating-frame state: (third-order y_new, y_new - embedded second order)."""
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(6)
    yn, err = np.zeros(6), np.zeros(6)
    lib().orc_bs3_single_step(ctypes.byref(pot), omega, h, _dp(y), _dp(yn), _dp(err))
    return yn, err


def jacobi_rot(pot: Pot, omega: float, y) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(6)
    return lib().orc_jacobi_rot(ctypes.byref(pot), omega, _dp(y))


def build_matrix_bs3(pot: Pot, omega: float, opts: BS3Opts, nsteps: int, ics: np.ndarray, obs: "Obs",
                     gh_v0s: Optional[np.ndarray] = None):
    """Orbit matrix (N, M) from the adaptive integrator: sample weights h_n / t_total
    (Sec. 2.2.4), shared by the mirror copies."""
    ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
    M = n_rows(obs)
    U = np.zeros((len(ics), M))
    drift = np.zeros(len(ics)); status = np.zeros(len(ics), dtype=np.int32)
    lib().orc_build_matrix_bs3(ctypes.byref(pot), omega, ctypes.byref(opts), nsteps, len(ics), _dp(ics),
                               ctypes.byref(obs), _gh_arg(obs, gh_v0s), _dp(U), _dp(drift),
                               status.ctypes.data_as(_I32))
    return U, drift, status


# ---------------------------------------------------------------------------
# Observables (Sec. 2.2.3-2.2.4)
# ---------------------------------------------------------------------------
def make_obs(g: dict) -> Obs:
    """Grid dict -> oracle struct.  Keys: incl, bar_angle, pa (radians), nx, ny,
    pix (pixel size, grid centred on the origin), nv, vmax, nR, nphi, nz, Rmax,
    zmin, zmax, gh, mirror4."""
    nx, ny, pix = g["nx"], g["ny"], g["pix"]
    nv = g.get("nv", 1)
    vmax = g.get("vmax", 400.0)
    return Obs(alpha=g.get("bar_angle", 0.0), beta=g["incl"], gamma=g.get("pa", 0.0),
               nx=nx, ny=ny, x0=-0.5 * nx * pix, y0=-0.5 * ny * pix, dx=pix, dy=pix,
               nv=nv, v0=-vmax, dv=2.0 * vmax / nv,
               nR=g["nR"], nphi=g["nphi"], nz=g["nz"], Rmax=g.get("Rmax", 10.0),
               zmin=g.get("zmin", -3.0), zmax=g.get("zmax", 3.0),
               gh=int(g.get("gh", 0)), mirror4=int(g.get("mirror4", 1)))


def euler_matrix(alpha: float, beta: float, gamma: float) -> np.ndarray:
    R = np.zeros(9)
    lib().orc_euler_matrix(alpha, beta, gamma, _dp(R))
    return R.reshape(3, 3)


def n_rows(obs: Obs) -> int:
    return lib().orc_n_rows(ctypes.byref(obs))


def row_blocks(obs: Obs) -> dict:
    nd = obs.nR * obs.nphi * obs.nz
    npix = obs.nx * obs.ny
    nk = 4 * npix if obs.gh else npix * obs.nv
    return {"dens": (0, nd), "pix": (nd, nd + npix), "kin": (nd + npix, nd + npix + nk)}


def build_matrix(pot: Pot, omega: float, dt: float, nsteps: int, ics: np.ndarray, obs: Obs,
                 gh_v0s: Optional[np.ndarray] = None):
    """Orbit matrix, orbit-major (N, M): row i is orbit i's column of U."""
    ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
    M = n_rows(obs)
    U = np.zeros((len(ics), M))
    drift = np.zeros(len(ics)); status = np.zeros(len(ics), dtype=np.int32)
    gh = _gh_arg(obs, gh_v0s)
    lib().orc_build_matrix(ctypes.byref(pot), omega, dt, nsteps, len(ics), _dp(ics), ctypes.byref(obs),
                           gh, _dp(U), _dp(drift), status.ctypes.data_as(_I32))
    return U, drift, status


def apply_matrix(pot: Pot, omega: float, dt: float, nsteps: int, ics: np.ndarray, obs: Obs, w: np.ndarray,
                 gh_v0s: Optional[np.ndarray] = None) -> np.ndarray:
    ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
    w = np.ascontiguousarray(w, dtype=np.float64)
    y = np.zeros(n_rows(obs))
    lib().orc_apply_matrix(ctypes.byref(pot), omega, dt, nsteps, len(ics), _dp(ics), ctypes.byref(obs),
                           _gh_arg(obs, gh_v0s), _dp(w), _dp(y))
    return y


def pixel_moments(pot: Pot, omega: float, dt: float, nsteps: int, ics: np.ndarray, obs: Obs,
                  w: np.ndarray) -> np.ndarray:
    ics = np.ascontiguousarray(ics, dtype=np.float64).reshape(-1, 6)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((obs.nx * obs.ny, 3))
    lib().orc_pixel_moments(ctypes.byref(pot), omega, dt, nsteps, len(ics), _dp(ics), ctypes.byref(obs),
                            _dp(w), _dp(out))
    return out


def gh_weights(w: float) -> np.ndarray:
    """2 sqrt(pi) alpha(w) H_m(w) for m = 0..4 (the per-sample GH row weights)."""
    out = np.zeros(5)
    lib().orc_gh_weights(w, _dp(out))
    return out


def _gh_arg(obs: Obs, gh_v0s):
    if not obs.gh:
        return None
    a = np.ascontiguousarray(gh_v0s, dtype=np.float64).reshape(-1, 2)
    assert len(a) == obs.nx * obs.ny
    return _dp(a)


def reduce_gh(U_orbit_major: np.ndarray, nd: int, npix: int, nv: int, vmin: float, dv: float,
              gh_v0s: np.ndarray) -> np.ndarray:
    """Velocity-histogram rows -> Gauss-Hermite rows: row (p, m) = sum_k
    U[(p, k)] * (2 sqrt(pi) alpha H_m)(w_k), w_k = (v_k - v0_p)/s_p at bin
    centres v_k (the GH weights of Eq. GH applied to the gridded LOSVD, as the
    paper's App. B does before comparing with data).  Input and output are
    orbit-major (N, rows)."""
    N = U_orbit_major.shape[0]
    out = np.zeros((N, nd + 5 * npix))
    out[:, :nd + npix] = U_orbit_major[:, :nd + npix]
    vc = vmin + (np.arange(nv) + 0.5) * dv
    for p in range(npix):
        v0, s = gh_v0s[p]
        W = np.array([gh_weights((v - v0) / s)[1:] for v in vc])          # (nv, 4)
        hist = U_orbit_major[:, nd + npix + p * nv: nd + npix + (p + 1) * nv]
        out[:, nd + npix + 4 * p: nd + npix + 4 * p + 4] = hist @ W
    return out


def bundle(U_orbit_major: np.ndarray, n: int) -> np.ndarray:
    """Orbit bundles (Sec. 2.2.1): the n dithered realisations of one initial
    condition enter the fit as one orbit, their mean column.  Input (N, rows)
    with the realisations of a bundle consecutive; output (N / n, rows)."""
    N, M = U_orbit_major.shape
    assert N % n == 0
    out = np.zeros((N // n, M))
    for k in range(n):
        out += U_orbit_major[k::n]
    return out / n


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return lib().orc_max_threads()


# ---------------------------------------------------------------------------
# Weight problem (Sec. 2.3): minimise 1/2 ||(U w - y)/sigma||^2 + (lam/N) ||w||^2, w >= 0
# ---------------------------------------------------------------------------
def whiten(U_rows: np.ndarray, y: np.ndarray, sigma: np.ndarray):
    """U_rows is (M, N).  Returns (U~, y~) = (diag(1/sigma) U, y / sigma)."""
    return U_rows / sigma[:, None], y / sigma


def normal_equations(Ut: np.ndarray, yt: np.ndarray, lam: float):
    """Objective 1/2 w^T H w - q^T w + const with H = U~^T U~ + (2 lam / N) I,
    q = U~^T y~ (Eq. objective_function in compact form)."""
    N = Ut.shape[1]
    H = Ut.T @ Ut + (2.0 * lam / N) * np.eye(N)
    q = Ut.T @ yt
    return H, q


def objective(H: np.ndarray, q: np.ndarray, w: np.ndarray) -> float:
    return 0.5 * w @ H @ w - q @ w


def nnls_lawson_hanson(A: np.ndarray, b: np.ndarray, tol: float = 1e-13, max_outer: int = 100000) -> np.ndarray:
    """Textbook Lawson-Hanson NNLS (Lawson & Hanson 1974, ch. 23): minimise
    ||A x - b|| subject to x >= 0, with the passive-set least-squares
    sub-problems solved by Householder QR (numpy lstsq)."""
    m, n = A.shape
    x = np.zeros(n)
    P = np.zeros(n, dtype=bool)
    wgrad = A.T @ (b - A @ x)
    scale = max(1.0, np.abs(wgrad).max())
    for _ in range(max_outer):
        Z = ~P
        if not Z.any() or wgrad[Z].max() <= tol * scale:
            break
        t = np.flatnonzero(Z)[np.argmax(wgrad[Z])]
        P[t] = True
        while True:
            z = np.zeros(n)
            z[P] = np.linalg.lstsq(A[:, P], b, rcond=None)[0]
            if np.all(z[P] > 0):
                x = z
                break
            bad = P & (z <= 0)
            alpha = np.min(x[bad] / (x[bad] - z[bad]))
            x = x + alpha * (z - x)
            P &= x > tol * max(1.0, np.abs(x).max())
            x[~P] = 0.0
        wgrad = A.T @ (b - A @ x)
    return x


def nnls_lh_normal(H: np.ndarray, q: np.ndarray, tol: float = 1e-13, max_outer: int = 1000000) -> np.ndarray:
    """The same Lawson-Hanson steps expressed on the normal equations
    (A^T A, A^T b) = (H, q): the passive-set sub-problem H_PP z_P = q_P is
    solved by Cholesky.  Minimises 1/2 x^T H x - q^T x subject to x >= 0."""
    n = len(q)
    x = np.zeros(n)
    P = np.zeros(n, dtype=bool)
    wgrad = q - H @ x
    scale = max(1.0, np.abs(q).max())
    for _ in range(max_outer):
        Z = ~P
        if not Z.any() or wgrad[Z].max() <= tol * scale:
            break
        t = np.flatnonzero(Z)[np.argmax(wgrad[Z])]
        P[t] = True
        while True:
            z = np.zeros(n)
            idx = np.flatnonzero(P)
            c = np.linalg.cholesky(H[np.ix_(idx, idx)])
            z[idx] = np.linalg.solve(c.T, np.linalg.solve(c, q[idx]))
            if np.all(z[P] > 0):
                x = z
                break
            bad = P & (z <= 0)
            alpha = np.min(x[bad] / (x[bad] - z[bad]))
            x = x + alpha * (z - x)
            P &= x > tol * max(1.0, np.abs(x).max())
            x[~P] = 0.0
        wgrad = q - H @ x
    return x


def nnls_bruteforce(H: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Enumerate every support S; the minimiser of the strictly convex problem
    is the feasible unconstrained minimiser on S with the lowest objective."""
    n = len(q)
    best, best_f = np.zeros(n), 0.0
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            z = np.linalg.solve(H[np.ix_(S, S)], q[S])
            if np.all(z >= 0):
                x = np.zeros(n); x[S] = z
                f = objective(H, q, x)
                if f < best_f:
                    best, best_f = x, f
    return best


def kkt_residual(H: np.ndarray, q: np.ndarray, w: np.ndarray) -> dict:
    """KKT certificate of min 1/2 w^T H w - q^T w, w >= 0: with g = H w - q,
    optimality is w >= 0, g >= 0, w_i g_i = 0.  Returns the violations and the
    projected gradient P(g) (g_i where w_i > 0, min(g_i, 0) where w_i = 0)."""
    g = H @ w - q
    pg = np.where(w > 0, g, np.minimum(g, 0.0))
    return {"neg_w": float(max(0.0, -w.min())), "neg_g": float(max(0.0, -g.min())),
            "compl": float(np.abs(w * g).max()), "pg_inf": float(np.abs(pg).max()),
            "pg_norm2": float(pg @ pg)}


def bootstrap_data(y: np.ndarray, sigma: np.ndarray, n_dens: int, xi: np.ndarray) -> np.ndarray:
    """Bootstrap realisations of the data (Sec. 2.4): every observed row (surface density
    and kinematics) perturbed by its error times a standard normal draw xi[b]; the
    3-D density rows (the first n_dens) are not bootstrapped.  Returns (B, M)."""
    Y = np.repeat(np.asarray(y, dtype=np.float64)[None, :], len(xi), axis=0)
    Y[:, n_dens:] += sigma[None, n_dens:] * xi[:, n_dens:]
    return Y


def chi2_model(chi2_b: np.ndarray) -> float:
    """Marginalised chi^2 over the bootstrap weight sets (Sec. 2.5): -2 ln of the
    bootstrap-averaged likelihood exp(-chi2_b / 2), evaluated relative to the smallest
    chi2_b so that no exponential over- or underflows:
    chi2_min - 2 ln[(1/B) sum_b exp(-(chi2_b - chi2_min) / 2)]."""
    c = np.asarray(chi2_b, dtype=np.float64)
    cmin = c.min()
    return float(cmin - 2.0 * np.log(np.mean(np.exp(-0.5 * (c - cmin)))))


def bootstrap_solve(U_rows: np.ndarray, y: np.ndarray, sigma: np.ndarray, lam: float, n_dens: int,
                    xi: np.ndarray):
    """One NNLS per bootstrap realisation with the same matrix (Lawson-Hanson on the
    normal equations, whose H is shared), and each weight set's observational chi^2
    against the observed data (density rows left out, Sec. 2.5).  Returns the weights
    (B, N), the chi2_b and the marginalised chi^2."""
    Yb = bootstrap_data(y, sigma, n_dens, xi)
    Ut = U_rows / sigma[:, None]
    H = Ut.T @ Ut + (2.0 * lam / U_rows.shape[1]) * np.eye(U_rows.shape[1])
    W = np.zeros((len(Yb), U_rows.shape[1]))
    chi = np.zeros(len(Yb))
    for b, yb in enumerate(Yb):
        W[b] = nnls_lh_normal(H, Ut.T @ (yb / sigma))
        r = (U_rows @ W[b] - y) / sigma
        chi[b] = float(r[n_dens:] @ r[n_dens:])
    return W, chi, chi2_model(chi)


def admm_nnls(H: np.ndarray, q: np.ndarray, rho: Optional[float] = None, tol: float = 1e-12,
              max_iter: int = 200000) -> tuple:
    """The paper's solver (Sec. 2.3): ADMM splitting into an unconstrained
    quadratic solve and a clip to w >= 0, with the scaled difference vector u
    carried between iterations.  FP64; Cholesky of H + rho I computed once."""
    n = len(q)
    if rho is None:
        rho = float(np.mean(np.diag(H)))
    c = np.linalg.cholesky(H + rho * np.eye(n))
    z = np.zeros(n); u = np.zeros(n)
    it = 0
    for it in range(1, max_iter + 1):
        rhs = q + rho * (z - u)
        w = np.linalg.solve(c.T, np.linalg.solve(c, rhs))
        z_prev = z
        z = np.maximum(0.0, w + u)
        u = u + w - z
        scale = max(1.0, np.abs(z).max())
        if np.abs(w - z).max() <= tol * scale and rho * np.abs(z - z_prev).max() <= tol * scale:
            break
    return z, it


def chi2_parts(U_rows: np.ndarray, y: np.ndarray, sigma: np.ndarray, w: np.ndarray, lam: float,
               n_dens: int) -> np.ndarray:
    """[chi2_total, chi2_obs, reg] (Sec. 2.3-2.4): chi2_total = ||(U w - y)/sigma||^2,
    chi2_obs leaves out the 3-D density rows (the first n_dens rows), and
    reg = (lam / N) ||w||^2."""
    r = (U_rows @ w - y) / sigma
    N = len(w)
    return np.array([float(r @ r), float(r[n_dens:] @ r[n_dens:]), lam / N * float(w @ w)])


# ---------------------------------------------------------------------------
# chi^2 emulator MLP (12 -> 256 -> 256 -> 256 -> 1, SiLU), FP64
# ---------------------------------------------------------------------------
def _sig(a):
    return 1.0 / (1.0 + np.exp(-a))


def mlp_forward(params: list, X: np.ndarray):
    """params = [W1, b1, W2, b2, W3, b3, W4, b4] with W_l of shape (out, in).
    Returns the output (B,) and the cache of pre-activations/activations."""
    h = X
    cache = [X]
    nl = len(params) // 2
    for l in range(nl):
        W, b = params[2 * l], params[2 * l + 1]
        a = h @ W.T + b
        if l < nl - 1:
            cache.append(a)
            h = a * _sig(a)
            cache.append(h)
        else:
            h = a
    return h[:, 0], cache


def mlp_loss_grad(params: list, X: np.ndarray, t: np.ndarray):
    """Mean-squared error and its gradient by hand-written back-propagation."""
    out, cache = mlp_forward(params, X)
    B = len(t)
    loss = float(np.mean((out - t) ** 2))
    d = (2.0 / B) * (out - t)[:, None]          # dL/d(output pre-activation)
    nl = len(params) // 2
    grads = [None] * len(params)
    for l in range(nl - 1, -1, -1):
        h_in = cache[2 * l]                      # input of layer l (X for l = 0)
        W = params[2 * l]
        grads[2 * l] = d.T @ h_in
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            a = cache[2 * l - 1]
            s = _sig(a)
            d = (d @ W) * (s * (1.0 + a * (1.0 - s)))
    return loss, grads


def adam_step(params: list, grads: list, m: list, v: list, t: int, lr: float = 1e-3,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """Adam (Kingma & Ba 2015) with bias correction, in place."""
    for k in range(len(params)):
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
