"""The paper's initial conditions (Sec. 2.2.1; h_R = 3.5, h_z = 1.2 kpc from
Sec. 3.2), generated on the host: positions from p(R, z) ~ R exp(-R/h_R)
exp(-|z|/h_z), velocities from the Jeans equations of that tracer in the
azimuthally averaged potential.

Pins: the position distribution's moments; the vertical Jeans integral in two
fields where it has a closed form; the azimuthal average of the bar against its
monopole far away and against the Miyamoto-Nagai potential it reduces to as the
needle shrinks; and equilibrium, checked with the oracle's integrator: in the
axisymmetric disc + halo the time-averaged occupancy of (R, z) cells over 2 Gyr
stays what the initial conditions fill, while the same positions with
velocities scaled by 0.8 or 1.25 drift far from it.
"""
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

G = inputs.G


def test_position_distribution():
    n, hR, hz = 20000, 3.5, 1.2
    ics = inputs.paper_ics(dict(inputs.DISC_HALO), n, 5)
    R = np.hypot(ics[:, 0], ics[:, 1])
    az = np.abs(ics[:, 2])
    assert abs(R.mean() - 2 * hR) < 4 * math.sqrt(2) * hR / math.sqrt(n)      # Gamma(2, h_R)
    assert abs(R.var() / (2 * hR * hR) - 1) < 0.05
    assert abs(az.mean() - hz) < 4 * hz / math.sqrt(n)                        # Exp(h_z)
    ph = np.arctan2(ics[:, 1], ics[:, 0])
    assert abs(np.cos(ph).mean()) < 0.03 and abs(np.sin(ph).mean()) < 0.03
    assert abs(np.mean(ics[:, 2] > 0) - 0.5) < 0.02
    assert np.all(np.isfinite(ics))


@pytest.mark.parametrize("z", [0.0, 0.7, 2.5])
def test_vertical_jeans_closed_forms(z):
    hR, hz = 3.0, 0.8
    R = np.array([4.0])
    # uniform vertical field Phi = g |z|: sigma_z^2 = g h_z
    g = 1500.0
    sR2, sz2, vp2, vc2 = inputs.jeans_moments(lambda a, b: g * np.abs(b), R, np.array([z]), hR, hz, beta_z=0.0)
    assert math.isclose(sz2[0], g * hz, rel_tol=1e-8)
    assert math.isclose(sR2[0], sz2[0], rel_tol=1e-12) and abs(vc2[0]) < 1e-6
    # no radial force and sigma_z independent of R: <v_phi^2> = sigma_z^2 (1 - R/h_R)
    assert math.isclose(vp2[0], sz2[0] * (1 - R[0] / hR), rel_tol=1e-6)
    # harmonic field Phi = k z^2 / 2 plus Omega^2 R^2 / 2: sigma_z^2 = k h_z (|z| + h_z), v_c^2 = Omega^2 R^2
    k, om2 = 900.0, 400.0
    beta = 0.3
    sR2, sz2, vp2, vc2 = inputs.jeans_moments(lambda a, b: 0.5 * k * b * b + 0.5 * om2 * a * a, R, np.array([z]),
                                              hR, hz, beta_z=beta)
    assert math.isclose(sz2[0], k * hz * (z + hz), rel_tol=1e-8)
    assert math.isclose(sR2[0], sz2[0] / (1 - beta), rel_tol=1e-12)
    assert math.isclose(vc2[0], om2 * R[0] ** 2, rel_tol=1e-6)
    assert math.isclose(vp2[0], sR2[0] * (1 - R[0] / hR) + om2 * R[0] ** 2, rel_tol=1e-6)


def test_azimuthally_averaged_bar():
    bar = dict(disc_M=0.0, disc_a=1.0, disc_b=1.0, bar_M=1e10, bar_L=4.0, bar_b=1.0, bar_c=0.5)
    far = inputs.axisym_potential(bar, np.array([300.0]), np.array([0.0]))[0]
    assert math.isclose(far, -G * 1e10 / 300.0, rel_tol=2e-4)
    short = dict(bar, bar_L=1e-4)
    R, z = np.array([0.5, 2.0, 7.0]), np.array([0.1, -1.0, 3.0])
    mn = -G * 1e10 / np.sqrt(R * R + (1.0 + np.sqrt(z * z + 0.25)) ** 2)
    np.testing.assert_allclose(inputs.axisym_potential(short, R, z), mn, rtol=1e-6)


def _occupancy_drift(orc, fac, n=10000, seed=77):
    p = dict(inputs.DISC_HALO)
    ics = inputs.paper_ics(p, n, seed)
    ics[:, 3:] *= fac
    grid = dict(nx=1, ny=1, pix=200.0, nv=1, vmax=1e4, incl=0.0, nR=12, nphi=1, nz=8, Rmax=24.0, zmin=-6.0,
                zmax=6.0)
    U, _, st = orc.build_matrix(orc.make_pot(p), 0.0, inputs.DT_HALF_MYR, 4000, ics, orc.make_obs(grid))
    assert (st != 0).sum() == 0
    avg = U[:, :96].sum(0) / n
    R, z = np.hypot(ics[:, 0], ics[:, 1]), ics[:, 2]
    H, _, _ = np.histogram2d(R, z, bins=[12, 8], range=[[0, 24], [-6, 6]])
    H = 0.5 * (H + H[:, ::-1]) / n                 # the mirror copies symmetrise z
    return np.abs(avg - H.ravel()).sum()


def test_jeans_initial_conditions_are_near_equilibrium(orc):
    eq = _occupancy_drift(orc, 1.0)
    cold, hot = _occupancy_drift(orc, 0.8), _occupancy_drift(orc, 1.25)
    assert eq < 0.12, eq
    assert cold > 2.0 * eq and hot > 2.0 * eq, (eq, cold, hot)
