"""Seeded synthetic inputs for the orbit-library hot path.

This module is the only code that both the CUDA path (through its callers) and
the FP64 oracle consume.  It draws random numbers and lays out workloads; it
computes none of the hot path's arithmetic (no force, integration, projection,
binning or solve).  Two small closed forms appear below only to SHAPE the
random initial conditions -- the Miyamoto-Nagai density for rejection sampling
and a disc+halo circular speed for the velocity scale -- and any other smooth
choice would serve; both sides then receive the identical ICs.

Units: kpc, km/s, Msun; one time unit is kpc/(km/s) = 977.79 Myr.

Workloads (the paper's scales: Sec. 2.2.1 7500 x 4 ICs, Sec. 2.2.2 5000 steps,
Sec. 3.1 ~600 apertures, Sec. 3.2.4 600 density cells, N_GH = 4):

* ``axisym_2k``   -- MN disc + NFW halo, no bar, Omega_p = 0; 2 000 orbits x
  2 000 steps; incl 60 deg; 20 x 20 pixels of 0.5 kpc x 16 velocity bins over
  +-400 km/s; 10 x 10 x 5 density cells (M = 7 300).  The small case the
  oracle finishes in seconds.
* ``barred_100k`` -- same disc and halo + Long-Murali bar (1e10 Msun, L = 4,
  a = 1, b = 0.5 kpc) rotating at Omega_p = 40 km/s/kpc; 100 000 orbits x
  10 000 steps; incl 45 deg, bar angle 30 deg; 50 x 50 pixels x 32 velocity
  bins; 20 x 20 x 10 cells (M = 86 500); 25 000 initial conditions drawn by the
  configurations' disc recipe (disc_ics) x 4 dithered realisations (orbit bundles).
* ``batched_64``  -- 64 trial potentials from a 12-D box, orbit counts
  U(10k, 100k), 5 000 steps; 30 x 20 pixels of 0.5 kpc (600 apertures, the
  paper's 60" x 40" field at 0.25 kpc/") with mass + GH h1..h4 rows, and
  10 x 12 x 5 = 600 density cells (M = 3 600).
* ``large_300k``  -- the barred potential; 300 000 orbits x 20 000 steps;
  60 x 60 pixels with mass + GH h1..h4 rows; 20 x 20 x 10 cells (M = 22 000);
  75 000 initial conditions from the paper's double-exponential disc with Jeans
  velocities (paper_ics, Sec. 2.2.1) x 4 dithered realisations.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

G = 4.300917e-6
KPC_KM = 3.0856775814913673e16
MYR_S = 3.15576e13
TIME_UNIT_MYR = KPC_KM / MYR_S          # 977.79 Myr
DT_HALF_MYR = 0.5 / TIME_UNIT_MYR        # 0.5 Myr in kpc/(km/s)
DEG = math.pi / 180.0

DISC_HALO = dict(disc_M=5e10, disc_a=3.0, disc_b=0.3, halo_M200=1e12, halo_c=10.0, H0=70.0)
BAR = dict(bar_M=1e10, bar_L=4.0, bar_b=1.0, bar_c=0.5)


def _grid(nx, ny, nv, nR, nphi, nz, incl, bar_angle=0.0, pa=0.0, gh=0, pix=0.5):
    return dict(nx=nx, ny=ny, pix=pix, nv=nv, vmax=400.0, nR=nR, nphi=nphi, nz=nz, Rmax=10.0,
                zmin=-3.0, zmax=3.0, incl=incl, bar_angle=bar_angle, pa=pa, gh=gh, mirror4=1)


WORKLOADS = {
    "axisym_2k": dict(potential=dict(DISC_HALO), omega_p=0.0, n_orb=2000, nsteps=2000, dt=DT_HALF_MYR,
                      grid=_grid(20, 20, 16, 10, 10, 5, 60 * DEG), seeds=dict(ic=1001, w=2001, noise=2002),
                      lam=1.0),
    "barred_100k": dict(potential=dict(DISC_HALO, **BAR), omega_p=40.0, n_orb=100_000, nsteps=10_000,
                        dt=DT_HALF_MYR, grid=_grid(50, 50, 32, 20, 20, 10, 45 * DEG, 30 * DEG),
                        seeds=dict(ic=1002, w=2001, noise=2002, dither=1003), lam=1.0, bundle=4, ics="disc"),
    "batched_64": dict(n_models=64, nsteps=5000, dt=DT_HALF_MYR, n_orb_range=(10_000, 100_000),
                       grid=_grid(30, 20, 40, 10, 12, 5, 0.0, gh=1), seeds=dict(box=3001, data=3100),
                       lam=1.0),
    "large_300k": dict(potential=dict(DISC_HALO, **BAR), omega_p=40.0, n_orb=300_000, nsteps=20_000,
                       dt=DT_HALF_MYR, grid=_grid(60, 60, 40, 20, 20, 10, 45 * DEG, 30 * DEG, gh=1),
                       seeds=dict(ic=1005, w=2001, noise=2002, dither=1006), lam=1.0, bundle=4, ics="paper"),
}

# 12-D trial box (disc M,a,b; bar M,L,b,c; Omega_p; halo M200,c; incl; bar angle).
# Masses log-uniform over x[0.5, 2] of the fiducial values.
BOX = dict(disc_M=(2.5e10, 1e11, "log"), disc_a=(2.0, 4.0, "lin"), disc_b=(0.2, 0.5, "lin"),
           bar_M=(5e9, 2e10, "log"), bar_L=(3.0, 5.0, "lin"), bar_b=(0.5, 1.5, "lin"), bar_c=(0.3, 0.8, "lin"),
           omega_p=(20.0, 60.0, "lin"), halo_M200=(5e11, 2e12, "log"), halo_c=(5.0, 20.0, "lin"),
           incl=(30 * DEG, 80 * DEG, "lin"), bar_angle=(0.0, 90 * DEG, "lin"))
BOX_KEYS = list(BOX.keys())


def rows_of(grid: dict) -> int:
    nd = grid["nR"] * grid["nphi"] * grid["nz"]
    npix = grid["nx"] * grid["ny"]
    return nd + npix + (4 * npix if grid.get("gh") else npix * grid["nv"])


def row_blocks(grid: dict) -> dict:
    nd = grid["nR"] * grid["nphi"] * grid["nz"]
    npix = grid["nx"] * grid["ny"]
    nk = 4 * npix if grid.get("gh") else npix * grid["nv"]
    return {"dens": (0, nd), "pix": (nd, nd + npix), "kin": (nd + npix, nd + npix + nk)}


# ---------------------------------------------------------------------------
# Initial conditions
# ---------------------------------------------------------------------------
def _mn_rho_shape(R, z, a, b):
    zeta = np.sqrt(z * z + b * b)
    c2 = R * R + (a + zeta) ** 2
    return (a * c2 + 3 * zeta * (a + zeta) ** 2) / (c2 ** 2.5 * zeta ** 3)


def _vcirc(R, z, p):
    """Circular speed of disc + halo at (R, z), used only to scale the random
    velocities."""
    a, b = p["disc_a"], p["disc_b"]
    zeta = np.sqrt(z * z + b * b)
    D2 = R * R + (a + zeta) ** 2
    dR = G * p["disc_M"] * R / D2 ** 1.5
    if p.get("halo_M200", 0.0) > 0:
        H = p.get("H0", 70.0) / 1000.0
        rho_c = 3 * H * H / (8 * math.pi * G)
        Rv = (3 * p["halo_M200"] / (4 * math.pi * 200 * rho_c)) ** (1.0 / 3.0)
        rs = Rv / p["halo_c"]
        Mdm = p["halo_M200"] / (math.log(1 + p["halo_c"]) - p["halo_c"] / (1 + p["halo_c"]))
        r = np.sqrt(R * R + z * z)
        s = r / rs
        dR = dR + G * Mdm * (np.log1p(s) - s / (1 + s)) / (r * r) * (R / r)
    return np.sqrt(np.maximum(R * dR, 0.0))


def disc_ics(p: dict, n: int, seed: int, Rmax: float = 20.0, zmax: float = 3.0,
             vfrac=(0.3, 1.1), sigma_v: float = 30.0) -> np.ndarray:
    """(n, 6) inertial ICs: positions rejection-sampled from the Miyamoto-Nagai
    disc density inside R < Rmax, |z| < zmax; velocities v_c U(0.3, 1.1) along
    +phi (prograde) plus isotropic Gaussian scatter sigma_v per component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a, b = p["disc_a"], p["disc_b"]
    rho_max = _mn_rho_shape(0.0, 0.0, a, b)
    out = []
    got = 0
    while got < n:
        m = max(4 * (n - got), 4096) * 32
        R = Rmax * np.sqrt(rng.random(m))
        ph = 2 * math.pi * rng.random(m)
        z = zmax * (2 * rng.random(m) - 1)
        keep = rng.random(m) * rho_max < _mn_rho_shape(R, z, a, b)
        R, ph, z = R[keep], ph[keep], z[keep]
        out.append(np.stack([R, ph, z], 1))
        got += len(R)
    Rpz = np.concatenate(out)[:n]
    R, ph, z = Rpz[:, 0], Rpz[:, 1], Rpz[:, 2]
    x, y = R * np.cos(ph), R * np.sin(ph)
    vc = _vcirc(R, z, p)
    f = vfrac[0] + (vfrac[1] - vfrac[0]) * rng.random(n)
    vt = vc * f
    vx = -vt * np.sin(ph) + sigma_v * rng.standard_normal(n)
    vy = vt * np.cos(ph) + sigma_v * rng.standard_normal(n)
    vz = sigma_v * rng.standard_normal(n)
    return np.ascontiguousarray(np.stack([x, y, z, vx, vy, vz], 1))


def workload_ics(p: dict, n: int, seed: int, kind: str = "disc") -> np.ndarray:
    """(n, 6) initial conditions of a workload: "disc" (disc_ics: the configurations' recipe of
    disc-density positions and scaled circular velocities) or "paper" (paper_ics: the paper's
    double-exponential disc with Jeans velocities, Sec. 2.2.1)."""
    if kind == "paper":
        return paper_ics(p, n, seed)
    if kind == "disc":
        return disc_ics(p, n, seed)
    raise ValueError(kind)


def dither(ics: np.ndarray, n: int, seed: int, p: dict, dx: float = 0.1, dv_frac: float = 0.05) -> np.ndarray:
    """Orbit bundles (Sec. 2.2.1): n nearby realisations of every initial condition,
    drawn uniformly from a box centred on it, dx kpc wide in each position and
    dv_frac v_c(R, z) wide in each velocity.  Returns (len(ics) * n, 6) inertial ICs,
    the n realisations of one bundle consecutive."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ics = np.asarray(ics, dtype=np.float64)
    R = np.hypot(ics[:, 0], ics[:, 1])
    vc = _vcirc(R, ics[:, 2], p)
    base = np.repeat(ics, n, axis=0)
    off = rng.random(base.shape) - 0.5
    off[:, :3] *= dx
    off[:, 3:] *= dv_frac * np.repeat(vc, n)[:, None]
    return np.ascontiguousarray(base + off)


# ---------------------------------------------------------------------------
# The paper's initial conditions (Sec. 2.2.1, with h_R = 3.5 and h_z = 1.2 kpc
# from Sec. 3.2): positions from p(R, z) ~ R exp(-R/h_R) exp(-|z|/h_z),
# velocities from the Jeans equations of that tracer in the azimuthally
# averaged potential (disc + halo + bar), drawn as Gaussians.
# ---------------------------------------------------------------------------
def _mn_phi(M, a, b, R, z):
    return -G * M / np.sqrt(R * R + (a + np.sqrt(z * z + b * b)) ** 2)


def _nfw_consts(p):
    H = p.get("H0", 70.0) / 1000.0
    rho_c = 3 * H * H / (8 * math.pi * G)
    Rv = (3 * p["halo_M200"] / (4 * math.pi * 200 * rho_c)) ** (1.0 / 3.0)
    c = p["halo_c"]
    return p["halo_M200"] / (math.log(1 + c) - c / (1 + c)), Rv / c


def _bar_phi(M, L, b, c, x, y, z):
    """Needle-convolved Miyamoto-Nagai bar (half-length L), with each log argument
    rationalised where its two terms would cancel."""
    Z = b + np.sqrt(z * z + c * c)
    q2 = y * y + Z * Z
    Tm = np.sqrt((L - x) ** 2 + q2)
    Tp = np.sqrt((L + x) ** 2 + q2)
    um, up = x - L, x + L
    num = np.where(um >= 0, um + Tm, q2 / np.maximum(Tm - um, 1e-300))
    den = np.where(up >= 0, up + Tp, q2 / np.maximum(Tp - up, 1e-300))
    return G * M / (2 * L) * np.log(num / den)


def axisym_potential(p: dict, R, z, n_phi: int = 32):
    """Disc + halo + the bar averaged over azimuth (trapezoid rule, exact for the
    bar's low azimuthal harmonics) at cylindrical (R, z)."""
    R = np.asarray(R, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    out = _mn_phi(p["disc_M"], p["disc_a"], p["disc_b"], R, z)
    if p.get("halo_M200", 0.0) > 0:
        Mdm, rs = _nfw_consts(p)
        r = np.maximum(np.sqrt(R * R + z * z), 1e-12)
        out = out - G * Mdm * np.log1p(r / rs) / r
    if p.get("bar_M", 0.0) > 0:
        ph = 2 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
        xs = R[..., None] * np.cos(ph)
        ys = R[..., None] * np.sin(ph)
        out = out + _bar_phi(p["bar_M"], p["bar_L"], p["bar_b"], p["bar_c"], xs, ys, z[..., None]).mean(-1)
    return out


def jeans_moments(phi_fn, R, z, h_R: float, h_z: float, beta_z: float = 0.2, n_quad: int = 40):
    """Second moments of a tracer nu ~ exp(-R/h_R - |z|/h_z) in an axisymmetric
    potential phi_fn(R, z), with a velocity ellipsoid aligned with the cylinder and
    sigma_R^2 = sigma_z^2 / (1 - beta_z):
      nu sigma_z^2 = int_|z|^inf nu dPhi/dz' dz'   (vertical equation; Gauss-Laguerre
                                                    in s = (z' - |z|)/h_z, exact weight),
      <v_phi^2> = b (sigma_z^2 + R d(nu sigma_z^2)/dR / nu) + R dPhi/dR,  b = 1/(1-beta_z).
    Returns (sigma_R^2, sigma_z^2, <v_phi^2>, v_c^2 = R dPhi/dR)."""
    R = np.asarray(R, dtype=np.float64)
    az = np.abs(np.asarray(z, dtype=np.float64))
    s, w = np.polynomial.laguerre.laggauss(n_quad)

    def sig2(RR):
        zq = az[..., None] + h_z * s
        d = 1e-4 * (1.0 + zq)
        fz = (phi_fn(RR[..., None], zq + d) - phi_fn(RR[..., None], zq - d)) / (2 * d)
        return h_z * (fz * w).sum(-1)

    dR = 1e-3 * (1.0 + R)
    s0 = sig2(R)
    ds = (sig2(R + dR) - sig2(np.maximum(R - dR, 0.0))) / (R + dR - np.maximum(R - dR, 0.0))
    fR = (phi_fn(R + dR, az) - phi_fn(np.maximum(R - dR, 0.0), az)) / (R + dR - np.maximum(R - dR, 0.0))
    vc2 = R * fR
    b = 1.0 / (1.0 - beta_z)
    vphi2 = b * (s0 + R * (ds - s0 / h_R)) + vc2
    return b * s0, s0, vphi2, vc2


def paper_ics(p: dict, n: int, seed: int, h_R: float = 3.5, h_z: float = 1.2, beta_z: float = 0.2,
              n_grid: int = 48) -> np.ndarray:
    """(n, 6) inertial initial conditions after Sec. 2.2.1: R ~ Gamma(2, h_R) and
    |z| ~ Exp(h_z) (the density p(R, z) ~ R exp(-R/h_R) exp(-|z|/h_z)), phi uniform;
    v_R, v_z ~ N(0, sigma_R), N(0, sigma_z); v_phi ~ N(vbar_phi, sigma_phi) with
    sigma_phi = sigma_R and vbar_phi = sqrt(<v_phi^2> - sigma_phi^2), the mean
    streaming the Jeans equations give (jeans_moments), tabulated on an
    n_grid x n_grid (R, |z|) grid and interpolated bilinearly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = rng.gamma(2.0, h_R, n)
    z = rng.exponential(h_z, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    ph = 2 * math.pi * rng.random(n)
    gR = np.concatenate([[0.0], np.geomspace(0.02, max(R.max(), 0.03) * 1.001, n_grid - 1)])
    gz = np.concatenate([[0.0], np.geomspace(0.01, max(np.abs(z).max(), 0.02) * 1.001, n_grid - 1)])
    RR, ZZ = np.meshgrid(gR, gz, indexing="ij")
    sR2, sz2, vp2, _ = jeans_moments(lambda a, b: axisym_potential(p, a, b), RR, ZZ, h_R, h_z, beta_z)
    sR2, sz2 = np.maximum(sR2, 0.0), np.maximum(sz2, 0.0)
    vbar2 = np.maximum(vp2 - sR2, 0.0)

    def interp(tab, x, y):
        i = np.clip(np.searchsorted(gR, x) - 1, 0, n_grid - 2)
        j = np.clip(np.searchsorted(gz, y) - 1, 0, n_grid - 2)
        tx = (x - gR[i]) / (gR[i + 1] - gR[i])
        ty = (y - gz[j]) / (gz[j + 1] - gz[j])
        return ((1 - tx) * (1 - ty) * tab[i, j] + tx * (1 - ty) * tab[i + 1, j] + (1 - tx) * ty * tab[i, j + 1]
                + tx * ty * tab[i + 1, j + 1])

    az = np.abs(z)
    sr, szz = np.sqrt(interp(sR2, R, az)), np.sqrt(interp(sz2, R, az))
    vbar = np.sqrt(interp(vbar2, R, az))
    vR = sr * rng.standard_normal(n)
    vz = szz * rng.standard_normal(n)
    vph = vbar + sr * rng.standard_normal(n)
    c, sn = np.cos(ph), np.sin(ph)
    return np.ascontiguousarray(np.stack([R * c, R * sn, z, vR * c - vph * sn, vR * sn + vph * c, vz], 1))


def plummer_ics(M: float, a: float, n: int, seed: int, rcut: float = 20.0) -> np.ndarray:
    """Plummer sphere from its isotropic distribution function f(E) ~ (-E)^(7/2)
    by the Aarseth, Henon & Wielen (1974) recipe (radii beyond rcut * a
    redrawn)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.empty(0)
    while len(r) < n:
        X = rng.random(2 * n) + 1e-300
        rr = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr < rcut * a]])
    r = r[:n]
    q = np.empty(0)
    while len(q) < n:
        x4 = rng.random(4 * n)
        x5 = 0.1 * rng.random(4 * n)
        q = np.concatenate([q, x4[x5 < x4 ** 2 * (1 - x4 ** 2) ** 3.5]])
    q = q[:n]
    vesc = np.sqrt(2 * G * M) * (r * r + a * a) ** -0.25
    v = q * vesc

    def iso(m):
        u = 2 * rng.random(m) - 1
        t = 2 * math.pi * rng.random(m)
        s = np.sqrt(1 - u * u)
        return np.stack([s * np.cos(t), s * np.sin(t), u], 1)

    pos = r[:, None] * iso(n)
    vel = v[:, None] * iso(n)
    return np.ascontiguousarray(np.concatenate([pos, vel], 1))


def kepler_ic(M: float, a: float, e: float) -> np.ndarray:
    """Pericentre of a Kepler ellipse in the x-y plane, moving along +y."""
    rp = a * (1 - e)
    vp = math.sqrt(G * M * (1 + e) / (a * (1 - e)))
    return np.array([rp, 0.0, 0.0, 0.0, vp, 0.0])


# ---------------------------------------------------------------------------
# Mock data recipe: w_true ~ U(0, 2); sigma_n = 2% max(y0_n, 1% of the row
# block's mean); y = y0 + sigma * N(0, 1).  The caller forms y0 = U w_true with
# whichever implementation it is testing against.
# ---------------------------------------------------------------------------
def true_weights(n: int, seed: int) -> np.ndarray:
    return 2.0 * np.random.Generator(np.random.PCG64(seed)).random(n)


def noise(m: int, seed: int) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(m)


def bootstrap_noise(m: int, n_boot: int, seed: int) -> np.ndarray:
    """(n_boot, m) standard normal draws for the bootstrap realisations of the data
    (Sec. 2.4: 100 realisations of the observed maps perturbed by their errors)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n_boot, m))


def mock_sigma(y0: np.ndarray, blocks: dict, frac: float = 0.02, gh_err: Optional[np.ndarray] = None) -> np.ndarray:
    """Errors per row.  Mass rows: frac * max(y0, 0.01 * block mean).  GH rows
    (when gh_err = per-pixel (dh1, dh2, dh3, dh4) is given): dh_m * Sigma_p with
    Sigma_p the pixel-mass row (the Rix et al. 1997 linearisation)."""
    s = np.zeros_like(y0)
    for name, (lo, hi) in blocks.items():
        if hi <= lo:
            continue
        if name == "kin" and gh_err is not None:
            plo, phi_ = blocks["pix"]
            sig_pix = np.maximum(y0[plo:phi_], 0.01 * max(y0[plo:phi_].mean(), 1e-300))
            s[lo:hi] = (gh_err * sig_pix[:, None]).reshape(-1)
        else:
            s[lo:hi] = frac * np.maximum(y0[lo:hi], 0.01 * max(y0[lo:hi].mean(), 1e-300))
    return s


def gh_reference(moments: np.ndarray, s_floor: float = 10.0, s_empty: float = 100.0):
    """Per-pixel reference Gaussian (v0, s) from mass-weighted moments
    (sum m, sum m v, sum m v^2), and the GH errors of Sec. 3.1:
    dh1 = 5/(sqrt2 s), dh2 = 5/(sqrt2 s), dh3 = dh4 = 0.03."""
    m0, m1, m2 = moments[:, 0], moments[:, 1], moments[:, 2]
    ok = m0 > 0
    v0 = np.where(ok, m1 / np.where(ok, m0, 1), 0.0)
    var = np.where(ok, m2 / np.where(ok, m0, 1) - v0 * v0, s_empty ** 2)
    s = np.where(ok, np.maximum(np.sqrt(np.maximum(var, 0.0)), s_floor), s_empty)
    v0s = np.ascontiguousarray(np.stack([v0, s], 1))
    err = np.stack([5 / (math.sqrt(2) * s), 5 / (math.sqrt(2) * s), np.full_like(s, 0.03), np.full_like(s, 0.03)], 1)
    return v0s, err


def draw_box(n: int, seed: int) -> np.ndarray:
    """n points of the 12-D trial box (columns in BOX_KEYS order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, len(BOX)))
    out = np.empty_like(u)
    for j, k in enumerate(BOX_KEYS):
        lo, hi, kind = BOX[k]
        out[:, j] = np.exp(np.log(lo) + u[:, j] * (np.log(hi) - np.log(lo))) if kind == "log" else lo + u[:, j] * (hi - lo)
    return out


def box_model(theta: np.ndarray) -> dict:
    """12-D box point -> (potential dict, omega_p, incl, bar_angle)."""
    d = {k: float(theta[j]) for j, k in enumerate(BOX_KEYS)}
    pot = dict(disc_M=d["disc_M"], disc_a=d["disc_a"], disc_b=d["disc_b"], halo_M200=d["halo_M200"],
               halo_c=d["halo_c"], H0=70.0, bar_M=d["bar_M"], bar_L=d["bar_L"], bar_b=d["bar_b"], bar_c=d["bar_c"])
    return dict(potential=pot, omega_p=d["omega_p"], incl=d["incl"], bar_angle=d["bar_angle"])


def box_unit(theta: np.ndarray) -> np.ndarray:
    """Map box points to [0, 1]^12 (log for masses) -- the surrogate's inputs."""
    theta = np.atleast_2d(theta)
    out = np.empty_like(theta, dtype=np.float64)
    for j, k in enumerate(BOX_KEYS):
        lo, hi, kind = BOX[k]
        out[:, j] = (np.log(theta[:, j]) - np.log(lo)) / (np.log(hi) - np.log(lo)) if kind == "log" else (theta[:, j] - lo) / (hi - lo)
    return out


def batched_orbit_counts(n_models: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_models)
