"""Pins for the oracle's fixed-step KDK integrator and Jacobi energy
(Sec. 2.2.2, with the fixed-dt symplectic step replacing Bogacki-Shampine).

Closed forms: the Kepler ellipse through Kepler's equation, a circular orbit
in the Miyamoto-Nagai plane; invariants: second-order convergence, time
reversibility, bounded (non-secular) energy and Jacobi-energy errors.
"""
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

G = 4.300917e-6


def kepler_position(M, a, e, t):
    """Position on the ellipse that starts at pericentre on +x moving along +y."""
    n = math.sqrt(G * M / a ** 3)
    Mm = n * t
    E = Mm
    for _ in range(60):
        E = E - (E - e * math.sin(E) - Mm) / (1 - e * math.cos(E))
    x = a * (math.cos(E) - e)
    y = a * math.sqrt(1 - e * e) * math.sin(E)
    return np.array([x, y, 0.0])


def test_kepler_ellipse_and_second_order(orc):
    M, a, e = 1e10, 2.0, 0.5
    pot = orc.make_pot(dict(test_kind=1, test_M=M))
    period = 2 * math.pi * math.sqrt(a ** 3 / (G * M))
    ic = inputs.kepler_ic(M, a, e)
    errs = []
    for nsteps in (2000, 4000, 8000):
        dt = 2 * period / nsteps
        tr = orc.trajectory(pot, 0.0, dt, nsteps, ic)
        exact = kepler_position(M, a, e, nsteps * dt)
        errs.append(np.linalg.norm(tr[-1, :3] - exact) / a)
    assert errs[0] < 1e-2
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 <= r1 <= 4.2 and 3.8 <= r2 <= 4.2, (errs, r1, r2)


def test_circular_orbit_in_mn_plane(orc):
    p = dict(disc_M=5e10, disc_a=3.0, disc_b=0.3)
    pot = orc.make_pot(p)
    R = 6.0
    _, acc = orc.potential(pot, np.array([[R, 0, 0]]), orc.DISC)
    vc = math.sqrt(R * -acc[0, 0])
    ic = np.array([R, 0, 0, 0, vc, 0])
    devs = []
    for dt in (4e-3, 2e-3):
        tr = orc.trajectory(pot, 0.0, dt, int(round(0.2 / dt)), ic)
        devs.append(np.abs(np.hypot(tr[:, 0], tr[:, 1]) - R).max() / R)
    assert devs[0] < 1e-2
    assert 3.5 < devs[0] / devs[1] < 4.5


def test_time_reversibility(orc):
    pot = orc.make_pot(dict(inputs.DISC_HALO, **inputs.BAR))
    ics = inputs.disc_ics(inputs.DISC_HALO, 4, seed=7)
    for ic in ics:
        S, dt = 1000, inputs.DT_HALF_MYR
        fw = orc.trajectory(pot, 0.0, dt, S, ic)
        back = fw[-1].copy(); back[3:] *= -1
        bw = orc.trajectory(pot, 0.0, dt, S, back)
        np.testing.assert_allclose(bw[-1, :3], ic[:3], atol=1e-10 * np.abs(ic[:3]).max())
        np.testing.assert_allclose(-bw[-1, 3:], ic[3:], atol=1e-10 * np.abs(ic[3:]).max())


def test_jacobi_bounded_with_rotating_bar(orc):
    """E_J is conserved by the exact flow in the rotating potential; the
    symplectic step keeps its error bounded, with no secular growth."""
    pot = orc.make_pot(dict(inputs.DISC_HALO, **inputs.BAR))
    ic = inputs.disc_ics(inputs.DISC_HALO, 1, seed=21, vfrac=(1.0, 1.0), sigma_v=5.0)[0]
    omega, dt, S = 40.0, inputs.DT_HALF_MYR, 40_000
    tr = orc.trajectory(pot, omega, dt, S, ic)
    ej = np.array([orc.jacobi(pot, omega, n * dt, tr[n]) for n in range(0, S + 1, 20)])
    rel = np.abs(ej - ej[0]) / abs(ej[0])
    half = len(rel) // 2
    assert rel.max() < 1e-4
    assert rel[half:].max() < 2.0 * rel[:half].max() + 1e-12


def test_drift_matches_trajectory_jacobi(orc):
    pot = orc.make_pot(dict(inputs.DISC_HALO, **inputs.BAR))
    ics = inputs.disc_ics(inputs.DISC_HALO, 3, seed=22)
    omega, dt, S = 40.0, inputs.DT_HALF_MYR, 300
    d = orc.drift(pot, omega, dt, S, ics)
    for i, ic in enumerate(ics):
        tr = orc.trajectory(pot, omega, dt, S, ic)
        ej = np.array([orc.jacobi(pot, omega, n * dt, tr[n]) for n in range(S + 1)])
        assert d[i] == pytest.approx(np.abs(ej[1:] - ej[0]).max() / abs(ej[0]), rel=1e-12)


def test_energy_bounded_static(orc):
    pot = orc.make_pot(dict(inputs.DISC_HALO))
    ic = inputs.disc_ics(inputs.DISC_HALO, 1, seed=23)[0]
    dt, S = inputs.DT_HALF_MYR, 20_000
    tr = orc.trajectory(pot, 0.0, dt, S, ic)
    e = np.array([orc.jacobi(pot, 0.0, 0.0, tr[n]) for n in range(0, S + 1, 10)])
    rel = np.abs(e - e[0]) / abs(e[0])
    assert rel.max() < 1e-4
    half = len(rel) // 2
    assert rel[half:].max() < 2.0 * rel[:half].max() + 1e-12
