"""Pins for the oracle's projection, mirroring and binning (Sec. 2.2.2 Table 1,
Sec. 2.2.3 Eq. Euler, Sec. 2.2.4, Eq. GH).

* hand-derived bins of a nearly static test particle (row layout, mirror signs,
  Euler convention, pixel / velocity / cylindrical indexing);
* rotation-matrix identities and the face-on / edge-on special cases;
* orthonormality of the Gauss-Hermite weights by Gauss-Hermite quadrature
  (a Gaussian LOSVD with the reference (v0, s) gives h0 = 1, h1..h4 = 0);
* the Plummer sphere's cell masses recovered by time-averaging orbits drawn
  from its own distribution function.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss

from paper_2607_00117_gb300 import inputs

DEG = math.pi / 180


def c1_obs(orc, **kw):
    g = dict(inputs.WORKLOADS["axisym_2k"]["grid"])
    g.update(kw)
    return orc.make_obs(g)


def test_hand_binned_particle(orc):
    """A test particle at (1.3, 0.7, 0.8) kpc moving at (0, 30, 20) km/s for four
    0.5 Myr steps (it moves 0.06 kpc in y and 0.04 in z; the 1 Msun point mass
    at the origin only keeps E_J finite).  With the axisym_2k grids (20 x 20
    pixels of 0.5 kpc from -5 kpc, 16 bins of 50 km/s from -400, 10 x 10 x 5
    cells over R < 10, phi in [0, 2 pi), z in [-3, 3)), incl 60 deg and
    alpha = gamma = 0, so X = x, Y = y/2 - (sqrt3/2) z, V = (sqrt3/2) v_y + v_z/2:

    copy (x,y,z):    ix 12, iy 9,  iv 8 (V = +36); iR 1, iphi 0, iz 3
    copy (x,y,-z):   ix 12, iy 12, iv 8 (V = +16); iR 1, iphi 0, iz 1
    copy (-x,-y,z):  ix 7,  iy 7,  iv 7 (V = -16); iR 1, iphi 5, iz 3
    copy (-x,-y,-z): ix 7,  iy 10, iv 7 (V = -36); iR 1, iphi 5, iz 1

    rows: density (iR*10 + iphi)*5 + iz; pixel 500 + iy*20 + ix; velocity
    900 + (iy*20 + ix)*16 + iv.  Each row collects 4 of the 16 sample copies.
    """
    pot = orc.make_pot(dict(test_kind=1, test_M=1.0))
    obs = c1_obs(orc)
    ic = np.array([[1.3, 0.7, 0.8, 0.0, 30.0, 20.0]])
    U, drift, status = orc.build_matrix(pot, 0.0, inputs.DT_HALF_MYR, 4, ic, obs)
    expected = {53: 0.25, 51: 0.25, 78: 0.25, 76: 0.25,
                500 + 192: 0.25, 500 + 252: 0.25, 500 + 147: 0.25, 500 + 207: 0.25,
                900 + 192 * 16 + 8: 0.25, 900 + 252 * 16 + 8: 0.25, 900 + 147 * 16 + 7: 0.25,
                900 + 207 * 16 + 7: 0.25}
    col = U[0]
    assert status[0] == 0
    got = {int(r): float(col[r]) for r in np.flatnonzero(col)}
    assert got == expected


def test_out_of_range_samples_dropped_but_pixel_mass_kept(orc):
    """Velocities beyond +-400 km/s leave the histogram but keep pixel mass."""
    pot = orc.make_pot(dict(test_kind=1, test_M=1.0))
    obs = c1_obs(orc)
    ic = np.array([[1.3, 0.7, 0.8, 0.0, 0.0, 900.0]])  # V = +-450 for every copy
    U, _, _ = orc.build_matrix(pot, 0.0, inputs.DT_HALF_MYR, 1, ic, obs)
    col = U[0]
    assert col[500:900].sum() == pytest.approx(1.0)
    assert col[900:].sum() == 0.0


def test_euler_matrix_identities(orc):
    rng = np.random.default_rng(3)
    for a, b, g in rng.random((20, 3)) * np.array([np.pi, np.pi / 2, np.pi]):
        R = orc.euler_matrix(a, b, g)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        # the disc normal's line-of-sight component is cos(inclination)
        assert R[2, 2] == pytest.approx(math.cos(b), abs=1e-14)
    # beta = 0 is face-on: v_los = v_z and the image is a rotation by alpha + gamma
    R = orc.euler_matrix(0.3, 0.0, 0.4)
    np.testing.assert_allclose(R[2], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(R[:2, :2], [[math.cos(0.7), -math.sin(0.7)], [math.sin(0.7), math.cos(0.7)]],
                               atol=1e-15)
    # beta = 90 deg with alpha = gamma = 0 is edge-on: v_los = v_y, Y = -z
    R = orc.euler_matrix(0.0, math.pi / 2, 0.0)
    np.testing.assert_allclose(R, [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-15)


def test_gh_weights_orthonormal(orc):
    """For a Gaussian LOSVD whose mean and dispersion equal the reference
    (v0, s), the per-sample weights integrate to h0 = 1 and h1..h4 = 0; and the
    weights of H_m times a Gaussian reproduce the orthonormality
    (1/sqrt pi) int exp(-x^2) H_m H_n = delta_mn."""
    x, wq = hermgauss(60)
    ws = np.sqrt(2.0) * x
    g = np.array([orc.gh_weights(w) for w in ws])            # (nodes, 5)
    h = (wq[:, None] * g).sum(0) / np.sqrt(np.pi)
    np.testing.assert_allclose(h, [1, 0, 0, 0, 0], atol=1e-13)
    # Gram matrix of H_m under exp(-x^2): (1/sqrt pi) sum wq H_m(x) H_n(x), with
    # H_m recovered from the weights at w = x by dividing out 2 sqrt(pi) alpha(x)
    gx_ = np.array([orc.gh_weights(w) for w in x])
    Hm = gx_ / (2 * np.sqrt(np.pi) * np.exp(-0.5 * x[:, None] ** 2) / np.sqrt(2 * np.pi))
    gram = (wq[:, None, None] * Hm[:, :, None] * Hm[:, None, :]).sum(0) / np.sqrt(np.pi)
    np.testing.assert_allclose(gram, np.eye(5), atol=1e-12)


def test_gh_rows_of_a_single_orbit(orc):
    """GH mode: row (p, m) of a particle that stays in one pixel equals the
    per-sample weight at its w = (V - v0)/s, averaged over copies."""
    pot = orc.make_pot(dict(test_kind=1, test_M=1.0))
    obs = c1_obs(orc, gh=1)
    npix = 400
    v0s = np.tile([5.0, 40.0], (npix, 1))
    ic = np.array([[1.3, 0.7, 0.8, 0.0, 30.0, 20.0]])
    U, _, _ = orc.build_matrix(pot, 0.0, inputs.DT_HALF_MYR, 1, ic, obs, gh_v0s=v0s)
    col = U[0]
    assert len(col) == 500 + 400 + 4 * 400
    # copy (x,y,z) at the first sample: pixel 192, V = (sqrt3/2) 30 + 20/2 (velocity
    # change over one step from the 1 Msun mass is < 1e-9 km/s)
    V = math.sqrt(3) / 2 * 30 + 10
    gw = orc.gh_weights((V - 5.0) / 40.0)
    np.testing.assert_allclose(col[900 + 4 * 192: 900 + 4 * 192 + 4], gw[1:] / 4, rtol=1e-9)


def test_plummer_density_recovered(orc):
    """Orbits drawn from the Plummer sphere's own DF and time-averaged give the
    sphere's mass in each cylindrical cell (within the sampling noise)."""
    M, a = 1e10, 1.0
    pot = orc.make_pot(dict(test_kind=2, test_M=M, test_a=a))
    g = dict(nx=2, ny=2, pix=1.0, nv=1, nR=4, nphi=2, nz=4, Rmax=2.0, zmin=-2.0, zmax=2.0, incl=0.0, gh=0,
             mirror4=1)
    obs = orc.make_obs(g)
    N = 3000
    ics = inputs.plummer_ics(M, a, N, seed=77)
    U, drift, status = orc.build_matrix(pot, 0.0, 1e-4, 1500, ics, obs)
    assert status.max() == 0 and drift.max() < 1e-3
    frac = U[:, :32].mean(0)
    # expected: cell mass / M, from quadrature of rho over R in [R0,R1], z in [z0,z1], phi share 1/2
    gx, gw = leggauss(40)
    exp = np.zeros(32)
    for iR in range(4):
        R0, R1 = 0.5 * iR, 0.5 * (iR + 1)
        for iz in range(4):
            z0, z1 = -2 + iz, -1 + iz
            Rq = 0.5 * (R1 - R0) * gx + 0.5 * (R1 + R0)
            zq = 0.5 * (z1 - z0) * gx + 0.5 * (z1 + z0)
            RR, ZZ = np.meshgrid(Rq, zq, indexing="ij")
            rho = 3 * M / (4 * np.pi * a ** 3) * (1 + (RR ** 2 + ZZ ** 2) / a ** 2) ** -2.5
            m = (np.outer(gw, gw) * rho * RR).sum() * 0.25 * (R1 - R0) * (z1 - z0) * np.pi
            for iphi in range(2):
                exp[(iR * 2 + iphi) * 4 + iz] = m / M
    sig = np.sqrt(exp / N)                 # Poisson bound per cell
    chi2 = (((frac - exp) / sig) ** 2).sum()
    assert chi2 / 32 < 2.0, chi2
    big = exp > 0.02
    np.testing.assert_allclose(frac[big], exp[big], rtol=0.08)


def test_recount_against_trajectory(orc):
    """Brute-force recount: re-bin every sample of the oracle's own trajectory
    with an independent loop and compare the density-cell counts."""
    p = dict(inputs.DISC_HALO, **inputs.BAR)
    pot = orc.make_pot(p)
    obs = c1_obs(orc)
    ics = inputs.disc_ics(inputs.DISC_HALO, 5, seed=5)
    S, omega, dt = 200, 40.0, inputs.DT_HALF_MYR
    U, _, _ = orc.build_matrix(pot, omega, dt, S, ics, obs)
    for i in range(len(ics)):
        tr = orc.trajectory(pot, omega, dt, S, ics[i])
        cnt = np.zeros(500)
        for n in range(1, S + 1):
            th = omega * (n * dt)
            c, s = math.cos(th), math.sin(th)
            x, y, z = tr[n, :3]
            xb, yb = c * x + s * y, -s * x + c * y
            for sx, sz in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
                X, Y, Z = sx * xb, sx * yb, sz * z
                R = math.hypot(X, Y)
                ph = math.atan2(Y, X) % (2 * math.pi)
                iR, iph, iz = int(R // 1.0), int(ph // (2 * math.pi / 10)), int((Z + 3) // 1.2)
                if iR < 10 and 0 <= iz < 5:
                    cnt[(iR * 10 + iph % 10) * 5 + iz] += 1
        np.testing.assert_allclose(U[i, :500] * 4 * S, cnt, atol=1e-9)


def test_reduce_gh_of_gaussian_histogram(orc):
    """A fine velocity histogram of a Gaussian LOSVD with the reference (v0, s)
    reduces to pixel mass m with GH rows (0, 0, 0, 0) * m, and a shifted
    Gaussian gives h1 of the sign of the shift (midpoint quadrature)."""
    nv, vmin, dv = 400, -400.0, 2.0
    vc = vmin + (np.arange(nv) + 0.5) * dv
    v0, s = 12.0, 55.0
    mass = 0.7
    hist = mass * np.exp(-0.5 * ((vc - v0) / s) ** 2) / (np.sqrt(2 * np.pi) * s) * dv
    U = np.concatenate([[0.3, mass], hist])[None, :]          # nd = 1, npix = 1
    out = orc.reduce_gh(U, 1, 1, nv, vmin, dv, np.array([[v0, s]]))
    np.testing.assert_allclose(out[0, :2], [0.3, mass])
    np.testing.assert_allclose(out[0, 2:], 0.0, atol=1e-9)
    out2 = orc.reduce_gh(U, 1, 1, nv, vmin, dv, np.array([[v0 - 10.0, s]]))
    assert out2[0, 2] > 0.05 * mass


def test_bundle_is_the_mean_of_consecutive_columns(orc):
    """Orbit bundles (Sec. 2.2.1): a hand case, identical realisations, and mass
    conservation (n x the bundle's column sum = the realisations' total)."""
    U = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0], [7.0, 9.0]])   # (N=4 orbits, 2 rows)
    np.testing.assert_array_equal(orc.bundle(U, 2), [[2.0, 3.0], [6.0, 7.5]])
    np.testing.assert_array_equal(orc.bundle(U, 1), U)
    rng = np.random.default_rng(5)
    col = rng.random(7)
    np.testing.assert_allclose(orc.bundle(np.tile(col, (3, 1)), 3), col[None, :], rtol=1e-15)
    V = rng.random((12, 5))
    B = orc.bundle(V, 4)
    np.testing.assert_allclose(4 * B.sum(axis=1), V.reshape(3, 4, 5).sum(axis=(1, 2)), rtol=1e-14)


def test_mirror_copies_follow_table1(orc):
    """Golden fixture: the sign patterns of Table 1 (Sec. 2.2.2).  A nearly free
    particle sampled once, viewed face-on (incl = 0, so X = x, Y = y, V = v_z
    of each copy), must land in the pixel, velocity and cylindrical bins that the
    table's signs give, each copy carrying 1/4 of the sample."""
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table1_mirrors.txt"))
    assert rows.shape == (4, 7)
    g = dict(nx=20, ny=20, pix=0.5, nv=16, vmax=400.0, nR=10, nphi=10, nz=5, Rmax=10.0, zmin=-3.0, zmax=3.0,
             incl=0.0, bar_angle=0.0, pa=0.0, gh=0, mirror4=1)
    pot = orc.make_pot(dict(test_kind=1, test_M=1e-6))
    ic = np.array([[1.3, 0.7, 0.8, 12.0, 30.0, 120.0]])
    U, _, status = orc.build_matrix(pot, 0.0, inputs.DT_HALF_MYR, 1, ic, orc.make_obs(g))
    assert status[0] == 0
    pos = ic[0, :3] + inputs.DT_HALF_MYR * ic[0, 3:]          # one drift step; the force is negligible
    vel = ic[0, 3:]
    nd, npix = 10 * 10 * 5, 20 * 20
    expected = {}
    for r in rows:
        sp, sv = r[1:4], r[4:7]
        x, y, z = sp * pos
        vz = (sv * vel)[2]
        ix, iy = int(math.floor((x + 5.0) / 0.5)), int(math.floor((y + 5.0) / 0.5))
        iv = int(math.floor((vz + 400.0) / 50.0))
        R, ph = math.hypot(x, y), math.atan2(y, x) % (2 * math.pi)
        iR, ip, iz = int(R / 1.0), int(ph / (2 * math.pi / 10)), int(math.floor((z + 3.0) / 1.2))
        p = iy * 20 + ix
        for row in ((iR * 10 + ip) * 5 + iz, nd + p, nd + npix + p * 16 + iv):
            expected[row] = expected.get(row, 0.0) + 0.25
    got = {int(k): float(U[0, k]) for k in np.flatnonzero(U[0])}
    assert got == expected
