"""Pins for the oracle's adaptive Bogacki-Shampine 3(2) integrator in the bar
frame (Sec. 2.2.2) and its step-weighted samples (Sec. 2.2.4).

Closed forms and invariants, each chosen so that a dropped term, a wrong sign or
a wrong coefficient fails it: third-order global convergence of the fixed-step
method and fourth- / third-order local errors of the solution and of its
embedded second-order estimate on the Kepler ellipse; the rotating-frame
equations (Coriolis and centrifugal terms, the frame change of the initial
condition and of the velocities) against the inertial Kepler solution; the
Jacobi energy conserved in the rotating barred potential and equal to its
inertial-frame form; every accepted step within the tolerance and the steps
shortest at pericentre; the sample weights h_n / t_total against the time an
eccentric Kepler orbit spends inside a radius (Kepler's equation).
"""
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

G = 4.300917e-6
M_K, A_K, E_K = 1e10, 2.0, 0.5


def kepler_state(M, a, e, t):
    """Position and velocity on the ellipse that starts at pericentre on +x moving along +y."""
    n = math.sqrt(G * M / a ** 3)
    Mm = n * t
    E = Mm
    for _ in range(60):
        E = E - (E - e * math.sin(E) - Mm) / (1 - e * math.cos(E))
    dE = n / (1 - e * math.cos(E))
    b = a * math.sqrt(1 - e * e)
    return np.array([a * (math.cos(E) - e), b * math.sin(E), 0.0, -a * math.sin(E) * dE, b * math.cos(E) * dE, 0.0])


def period(M, a):
    return 2 * math.pi * math.sqrt(a ** 3 / (G * M))


@pytest.fixture(scope="module")
def kep(orc):
    return orc.make_pot(dict(test_kind=1, test_M=M_K))


def test_fixed_step_third_order_on_kepler(orc, kep):
    ic = inputs.kepler_ic(M_K, A_K, E_K)
    P = period(M_K, A_K)
    errs = []
    for n in (1000, 2000, 4000):
        h = 2 * P / n
        ts, ys, rej = orc.bs3_trajectory(kep, 0.0, orc.bs3_opts(h0=h, fixed=True), n, ic)
        assert rej == 0 and math.isclose(ts[-1], 2 * P, rel_tol=1e-12)
        errs.append(np.linalg.norm(ys[-1, :3] - kepler_state(M_K, A_K, E_K, ts[-1])[:3]) / A_K)
    assert errs[0] < 1e-3
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 <= r1 <= 9.0 and 7.0 <= r2 <= 9.0, (errs, r1, r2)


def test_local_errors_of_the_pair(orc, kep):
    """One step from pericentre: the third-order solution's local error falls as
    h^4, the embedded difference (a second-order local error) as h^3."""
    y0 = inputs.kepler_ic(M_K, A_K, E_K)
    P = period(M_K, A_K)
    loc, est = [], []
    for h in (P / 200, P / 400, P / 800):
        yn, err = orc.bs3_single_step(kep, 0.0, h, y0)
        loc.append(np.linalg.norm(yn[:3] - kepler_state(M_K, A_K, E_K, h)[:3]))
        est.append(np.linalg.norm(err[:3]))
    for k in range(2):
        assert 14.0 <= loc[k] / loc[k + 1] <= 18.0, loc
        assert 7.0 <= est[k] / est[k + 1] <= 9.0, est


def test_rotating_frame_against_inertial_kepler(orc, kep):
    """In the frame rotating at Omega_p = 40 km/s/kpc the point-mass orbit is no
    longer an ellipse; mapped back to the inertial frame it must be, with the
    inertial velocity.  A sign error in the Coriolis or centrifugal term, or in
    either frame change, moves it by O(1)."""
    ic = inputs.kepler_ic(M_K, A_K, E_K)
    P = period(M_K, A_K)
    n = 4000
    ts, ys, _ = orc.bs3_trajectory(kep, 40.0, orc.bs3_opts(h0=P / n, fixed=True), n, ic)
    inert = orc.rotating_to_inertial(40.0, ts, ys)
    exact = np.array([kepler_state(M_K, A_K, E_K, t) for t in ts])
    v0 = np.linalg.norm(ic[3:])
    assert np.abs(inert[:, :3] - exact[:, :3]).max() < 1e-6 * A_K
    assert np.abs(inert[:, 3:] - exact[:, 3:]).max() < 1e-6 * v0
    # the rotating-frame state itself is far from the inertial one
    assert np.abs(ys[n // 2, :3] - exact[n // 2, :3]).max() > 0.1 * A_K


def test_jacobi_energy_in_the_rotating_bar(orc):
    pot = orc.make_pot(dict(inputs.DISC_HALO, **inputs.BAR))
    omega = 40.0
    ic = inputs.disc_ics(inputs.DISC_HALO, 1, seed=21, vfrac=(1.0, 1.0), sigma_v=5.0)[0]
    ts, ys, _ = orc.bs3_trajectory(pot, omega, orc.bs3_opts(h0=inputs.DT_HALF_MYR / 4, fixed=True), 4000, ic)
    ej = np.array([orc.jacobi_rot(pot, omega, y) for y in ys])
    assert np.abs(ej / ej[0] - 1).max() < 5e-8
    # the rotating-frame expression equals the inertial one at the same instant
    inert = orc.rotating_to_inertial(omega, ts, ys)
    for k in (0, 1000, 4000):
        assert math.isclose(orc.jacobi(pot, omega, ts[k], inert[k]), ej[k], rel_tol=1e-12)
    # adaptive at the paper's tolerance: drift of the order the paper reports
    # (1e-4 to 1e-2 over 5 000 steps), smaller at a tighter tolerance
    drifts = []
    for rtol in (1e-4, 1e-6):
        _, yy, rej = orc.bs3_trajectory(pot, omega, orc.bs3_opts(rtol=rtol), 5000, ic)
        assert rej >= 0
        e = np.array([orc.jacobi_rot(pot, omega, y) for y in yy])
        drifts.append(np.abs(e / e[0] - 1).max())
    assert drifts[0] < 1e-2 and drifts[1] < 0.1 * drifts[0], drifts


def test_accepted_steps_meet_the_tolerance(orc, kep):
    ic = inputs.kepler_ic(M_K, A_K, E_K)
    rtol = 1e-5
    ts, ys, rej = orc.bs3_trajectory(kep, 0.0, orc.bs3_opts(rtol=rtol), 3000, ic)
    assert rej >= 0
    h = np.diff(ts)
    for k in range(0, 3000, 97):
        yn, err = orc.bs3_single_step(kep, 0.0, h[k], ys[k])
        np.testing.assert_allclose(yn, ys[k + 1], rtol=1e-12, atol=1e-12)   # the step that was taken
        sx = rtol * max(np.linalg.norm(ys[k, :3]), np.linalg.norm(yn[:3]))
        sv = rtol * max(np.linalg.norm(ys[k, 3:]), np.linalg.norm(yn[3:]))
        assert max(np.linalg.norm(err[:3]) / sx, np.linalg.norm(err[3:]) / sv) <= 1.0
    # steps follow the orbit: shortest at pericentre, longest at apocentre
    r = np.linalg.norm(ys[1:, :3], axis=1)
    peri, apo = h[r < A_K * (1 - E_K) * 1.05], h[r > A_K * (1 + E_K) * 0.95]
    assert apo.mean() / peri.mean() > 3.0, (apo.mean(), peri.mean())


def test_sample_weights_follow_time_on_an_eccentric_orbit(orc, kep):
    """Sample n carries h_n / t_total: the weight in radial cells inside r0 equals
    the fraction of time the Kepler orbit spends inside r0, (E0 - e sin E0) / pi
    with cos E0 = (1 - r0/a) / e.  Equal weights 1/S would overweight the short
    pericentre steps (checked too)."""
    ic = inputs.kepler_ic(M_K, A_K, E_K)
    S = 5000
    grid = dict(nx=1, ny=1, pix=100.0, nv=1, vmax=1e4, incl=0.0, nR=40, nphi=1, nz=1, Rmax=4.0, zmin=-1.0, zmax=1.0)
    obs = orc.make_obs(grid)
    opts = orc.bs3_opts(rtol=1e-4)
    U, drift, status = orc.build_matrix_bs3(kep, 0.0, opts, S, ic[None, :], obs)
    assert status[0] == 0
    dens = U[0, :40]
    assert math.isclose(dens.sum(), 1.0, rel_tol=1e-12)          # every sample inside the cells
    assert math.isclose(U[0, 40], 1.0, rel_tol=1e-12)            # and inside the one pixel
    ts, ys, _ = orc.bs3_trajectory(kep, 0.0, opts, S, ic)
    n_periods = ts[-1] / period(M_K, A_K)
    assert n_periods > 30
    edges = np.arange(1, 41) * 0.1
    cum = np.cumsum(dens)
    r_eq = np.linalg.norm(ys[1:, :3], axis=1)
    worst, worst_eq = 0.0, 0.0
    for k, r0 in enumerate(edges):
        if not (A_K * (1 - E_K) < r0 < A_K * (1 + E_K)):
            continue
        E0 = math.acos((1 - r0 / A_K) / E_K)
        frac = (E0 - E_K * math.sin(E0)) / math.pi
        worst = max(worst, abs(cum[k] - frac))
        worst_eq = max(worst_eq, abs(np.mean(r_eq < r0) - frac))
    assert worst < 1.5 / n_periods + 0.01, worst
    assert worst_eq > 0.1, worst_eq


def test_sampled_velocities_are_inertial(orc, kep):
    """A circular point-mass orbit integrated in the frame rotating at 40 km/s/kpc
    and seen edge-on (line of sight along the bar frame's y axis): the sampled
    velocity is the inertial one in bar axes, of constant length v_c and uniformly
    distributed direction, so <V^2> = v_c^2 / 2 over the step-weighted samples.
    The rotating-frame velocity (v_c - Omega R in length) would give about 80 % less."""
    R0 = 2.0
    vc = math.sqrt(G * M_K / R0)
    ic = np.array([R0, 0.0, 0.0, 0.0, vc, 0.0])
    grid = dict(nx=1, ny=1, pix=100.0, nv=200, vmax=400.0, incl=math.pi / 2, nR=1, nphi=1, nz=1, Rmax=10.0,
                zmin=-1.0, zmax=1.0)
    obs = orc.make_obs(grid)
    U, _, status = orc.build_matrix_bs3(kep, 40.0, orc.bs3_opts(rtol=1e-6), 4000, ic[None, :], obs)
    assert status[0] == 0
    hist = U[0, 2:]
    assert math.isclose(hist.sum(), 1.0, rel_tol=1e-12)
    centres = -400.0 + (np.arange(200) + 0.5) * 4.0
    v2 = float(hist @ centres ** 2)
    assert abs(v2 / (0.5 * vc * vc) - 1.0) < 0.01, (v2, 0.5 * vc * vc)
