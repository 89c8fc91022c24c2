"""GPU parity of the orbit-library path (potential, KDK integration, Jacobi
drift, mirrors, projection, binning, GH rows) against the FP64 oracle, through
the C-ABI.

Gates (stated for this method): integer bin counts bit-exact over the first
64 steps (FP64 form; the FP32 form exact outside a 1e-5 bin-width guard band
around bin edges); per-step phase-space error <= 1e-5 relative over 1e3 steps
for regular orbits (FP32 form against FP64); orbit-matrix L1 difference
<= 1e-3 per orbit.

Two readings make the FP32 gates well posed.  "Regular" means a twin orbit
displaced by 1e-9 kpc separates by less than 1e4 x over the 1e3 steps; any
other orbit is held to the oracle's own spread under perturbations of its
initial condition (FP32 rounding of each step's force is ~1e-7 relative and
accumulates to a few 1e-6 over 1e3 steps on regular orbits).  The per-orbit matrix gate allows, on top of
1e-3, the moves of sample copies whose oracle coordinate lies within 2e-4
bin widths of an edge (guard band, counted from the oracle trajectory); orbits
whose oracle column itself moves by > 2e-4 under a 1e-7 relative change of the
initial conditions are excluded, counted, and must stay a small minority.
"""
from _guard import guard_events
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

W1 = inputs.WORKLOADS["axisym_2k"]
W2 = inputs.WORKLOADS["barred_100k"]
BARRED = dict(inputs.DISC_HALO, **inputs.BAR)
# the paper's bar (Sec. 2.1.2): Dehnen-Aly T3 long bar + V4 bulge of total mass M_b, half-length L_b
PAPER_BAR = dict(inputs.DISC_HALO, bar_M=1e10, bar_L=4.0, bar_kind=1)


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    return swmod


def ctx_for(sw, prec, pot):
    c = sw.Context(0, prec)
    c.set_potential(pot)
    return c


def test_potential_and_force(sw, orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 5, (400, 3)), rng.normal(0, 30, (100, 3)),
                        np.array([[4.0, 0, 0], [-4, 0.01, 0], [0, 0, 0.001], [1e-4, 1e-4, 0]])])
    pot = orc.make_pot(BARRED)
    phi_o, acc_o = orc.potential(pot, x)
    for prec, rtol in (("fp64", 1e-12), ("fp32", 3e-6)):
        c = ctx_for(sw, prec, BARRED)
        phi, acc = c.potential_eval(x)
        np.testing.assert_allclose(phi, phi_o, rtol=rtol)
        scale = np.linalg.norm(acc_o, axis=1, keepdims=True)
        assert np.all(np.abs(acc - acc_o) <= rtol * 4 * scale + 1e-30), prec


def test_potential_and_force_paper_bar(sw, orc):
    """The paper's Dehnen-Aly T3 + V4 bar (bar_kind 1) with the disc and halo, and the bar
    alone, at 1e3 points against the oracle (its needle integrals by 48-point quadrature):
    FP64 to 1e-11; FP32 potential to 1e-6 (total) and 3e-5 (bar alone), force to 5e-5 and
    3e-4 of |a| floored at 1e-3 of the median |a| (it vanishes at the centre, where only an
    absolute error means anything).  The bar alone is looser in FP32: far from the needle
    its closed forms take differences of nearly equal antiderivatives, a loss that is small
    against the total force there."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 3, (500, 3)), rng.normal(0, 12, (494, 3)),
                        np.array([[0.0, 0, 0], [4.0, 0, 0], [-4.0, 0.01, 0], [0.05, 0, 0.02],
                                  [30.0, -20.0, 5.0], [1e-4, 1e-4, 0]])])
    bar_only = dict(disc_M=0.0, disc_a=3.0, disc_b=0.3, halo_M200=0.0, halo_c=10.0, bar_M=1e10, bar_L=4.0,
                    bar_kind=1)
    for pot, tol32 in ((PAPER_BAR, (1e-6, 5e-5)), (bar_only, (3e-5, 3e-4))):
        phi_o, acc_o = orc.potential(orc.make_pot(pot), x)
        n = np.linalg.norm(acc_o, axis=1, keepdims=True)
        scale = np.maximum(n, 1e-3 * np.median(n))
        for prec, (tp, ta) in (("fp64", (1e-11, 1e-11)), ("fp32", tol32)):
            c = ctx_for(sw, prec, pot)
            phi, acc = c.potential_eval(x)
            np.testing.assert_allclose(phi, phi_o, rtol=tp)
            assert np.all(np.abs(acc - acc_o) <= ta * scale), (prec, (np.abs(acc - acc_o) / scale).max())
    c = sw.Context(0, "fp32")
    with pytest.raises(sw.SwError):
        c.set_potential(dict(PAPER_BAR, bar_kind=2))


def _grid(W, **kw):
    g = dict(W["grid"]); g.update(kw)
    return g


def _counts(U, S, ncopy=4):
    return np.rint(U * ncopy * S).astype(np.int64)


@pytest.mark.parametrize("pot_name", ["axisym", "barred", "paper_bar"])
def test_counts_bit_exact_64_steps_fp64(sw, orc, pot_name):
    pot = {"axisym": inputs.DISC_HALO, "barred": BARRED, "paper_bar": PAPER_BAR}[pot_name]
    omega = 0.0 if pot_name == "axisym" else 40.0
    grid = _grid(W1) if pot_name == "axisym" else _grid(W2, nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    ics = inputs.disc_ics(inputs.DISC_HALO, 700, seed=101)     # several 128-orbit tiles + ragged tail
    S, dt = 64, inputs.DT_HALF_MYR
    c = ctx_for(sw, "fp64", pot)
    c.integrate_library(ics, omega, dt, S)
    U = c.project(grid)
    Ug = U.copy()
    Uo, drift_o, status_o = orc.build_matrix(orc.make_pot(pot), omega, dt, S, ics, orc.make_obs(grid))
    np.testing.assert_array_equal(_counts(Ug, S), _counts(Uo, S))
    assert np.abs(Ug - Uo).max() <= 1e-15
    drift_g, status_g = c.project_stats(len(ics))
    np.testing.assert_array_equal(status_g, status_o)
    np.testing.assert_allclose(drift_g, drift_o, rtol=1e-6, atol=1e-13)


def test_counts_fp32_outside_guard_band(sw, orc):
    """FP32 form: counts equal the oracle's except for samples whose oracle
    coordinate lies within 1e-5 bin widths of a bin edge."""
    pot, omega = BARRED, 40.0
    grid = _grid(W2, nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    ics = inputs.disc_ics(inputs.DISC_HALO, 300, seed=102)
    S, dt = 64, inputs.DT_HALF_MYR
    c = ctx_for(sw, "fp32", pot)
    c.integrate_library(ics, omega, dt, S)
    Ug = c.project(grid).copy()
    Uo, _, _ = orc.build_matrix(orc.make_pot(pot), omega, dt, S, ics, orc.make_obs(grid))
    diff = np.abs(_counts(Ug, S) - _counts(Uo, S)).sum(axis=1)
    # guard-band samples per orbit from the oracle trajectory
    R = orc.euler_matrix(grid["bar_angle"], grid["incl"], grid.get("pa", 0.0))
    band = 1e-5
    near = np.zeros(len(ics), dtype=int)
    for i, ic in enumerate(ics):
        tr = orc.trajectory(orc.make_pot(pot), omega, dt, S, ic)[1:]
        th = omega * dt * np.arange(1, S + 1)
        cth, sth = np.cos(th), np.sin(th)
        xb = cth * tr[:, 0] + sth * tr[:, 1]; yb = -sth * tr[:, 0] + cth * tr[:, 1]; zb = tr[:, 2]
        vxb = cth * tr[:, 3] + sth * tr[:, 4]; vyb = -sth * tr[:, 3] + cth * tr[:, 4]; vzb = tr[:, 5]
        for sx, sz in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
            p = np.stack([sx * xb, sx * yb, sz * zb]); v = np.stack([sx * vxb, sx * vyb, sz * vzb])
            X, Y, V = R[0] @ p, R[1] @ p, R[2] @ v
            coords = [(X + 5.0) / 0.5, (Y + 5.0) / 0.5, (V + 400.0) / 50.0, np.hypot(p[0], p[1]) / 1.0,
                      (np.arctan2(p[1], p[0]) % (2 * np.pi)) / (2 * np.pi / 10), (p[2] + 3.0) / 1.2]
            for u in coords:
                near[i] += int(np.sum(np.abs(u - np.rint(u)) < band))
    assert np.all(diff <= 2 * near), (np.flatnonzero(diff > 2 * near), diff[diff > 2 * near])
    assert diff.sum() <= max(4, 2 * near.sum())


def test_phase_space_fp32_regular_orbits(sw, orc):
    """Per-step relative error <= 1e-5 over 1e3 steps for regular orbits.  An
    orbit is regular if a twin displaced by 1e-9 kpc separates by less than
    1e4 x over the same steps (oracle FP64).  The error at each step is relative
    to the orbit's own scale: |dx(t)| / max_t |x| and |dv(t)| / max_t |v| (a
    pointwise |v(t)| near a turning point would measure a phase error against a
    vanishing speed).  Every other orbit is held to the oracle's own spread: its
    error at each step is at most 3 x the largest deviation of the oracle's
    trajectory under four seeded relative perturbations of 1e-6 of its initial
    condition, plus 1e-5."""
    pot, omega = BARRED, 40.0
    ics = inputs.disc_ics(inputs.DISC_HALO, 64, seed=103)
    S, dt = 1000, inputs.DT_HALF_MYR
    po = orc.make_pot(pot)
    c = ctx_for(sw, "fp32", pot)
    tg = c.trajectory(ics, omega, dt, S)
    n_regular, n_spread, worst = 0, 0, 0.0
    for i, ic in enumerate(ics):
        to = orc.trajectory(po, omega, dt, S, ic)
        ic2 = ic.copy(); ic2[0] += 1e-9
        t2 = orc.trajectory(po, omega, dt, S, ic2)
        amp = np.linalg.norm(t2[:, :3] - to[:, :3], axis=1).max() / 1e-9
        sx = np.linalg.norm(to[:, :3], axis=1).max()
        sv = np.linalg.norm(to[:, 3:], axis=1).max()
        err = np.maximum(np.linalg.norm(tg[i, :, :3] - to[:, :3], axis=1) / sx,
                         np.linalg.norm(tg[i, :, 3:] - to[:, 3:], axis=1) / sv)
        if amp < 1e4:
            n_regular += 1
            worst = max(worst, err.max())
            assert err.max() <= 1e-5, (i, amp, err.max())
        else:
            n_spread += 1
            spread = np.zeros(S + 1)
            rng = np.random.default_rng(6100 + i)
            for _ in range(4):
                tp = orc.trajectory(po, omega, dt, S, ic * (1 + 1e-6 * rng.standard_normal(6)))
                spread = np.maximum(spread, np.maximum(np.linalg.norm(tp[:, :3] - to[:, :3], axis=1) / sx,
                                                       np.linalg.norm(tp[:, 3:] - to[:, 3:], axis=1) / sv))
            assert np.all(err <= 3 * spread + 1e-5), (i, amp, err.max(), spread.max())
    print(f"phase space: {n_regular} regular orbits (largest error {worst:.3g}), {n_spread} under the spread gate")
    assert n_regular + n_spread == len(ics) and n_regular >= len(ics) // 2


def test_phase_space_fp64(sw, orc):
    pot, omega = BARRED, 40.0
    ics = inputs.disc_ics(inputs.DISC_HALO, 8, seed=104)
    S, dt = 1000, inputs.DT_HALF_MYR
    c = ctx_for(sw, "fp64", pot)
    tg = c.trajectory(ics, omega, dt, S)
    for i, ic in enumerate(ics):
        to = orc.trajectory(orc.make_pot(pot), omega, dt, S, ic)
        np.testing.assert_allclose(tg[i, :100], to[:100], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matrix_l1_axisym_2k(sw, orc, prec):
    """Full axisym_2k workload (2000 orbits x 2000 steps): per-orbit L1 of the
    matrix difference <= 1e-3 (columns sum to <= 3 here: density + pixel +
    velocity rows)."""
    W = W1
    ics = inputs.disc_ics(W["potential"], W["n_orb"], seed=W["seeds"]["ic"])
    c = ctx_for(sw, prec, W["potential"])
    c.integrate_library(ics, W["omega_p"], W["dt"], W["nsteps"])
    Ug = c.project(W["grid"]).copy()
    Uo, _, so = orc.build_matrix(orc.make_pot(W["potential"]), W["omega_p"], W["dt"], W["nsteps"], ics,
                                 orc.make_obs(W["grid"]))
    l1 = np.abs(Ug - Uo).sum(axis=1)
    if prec == "fp64":
        assert l1.max() <= 1e-3, (prec, l1.max(), np.argmax(l1))
        return
    allow = _allowance(orc, W["potential"], W["omega_p"], W["dt"], W["nsteps"], ics, W["grid"], l1 > 1e-3,
                       per_event=2.0 / (4 * W["nsteps"]))
    bad = l1 > 1e-3 + allow
    stable = _stable_columns(orc, W["potential"], W["omega_p"], W["dt"], W["nsteps"], ics, W["grid"], Uo, bad)
    assert np.all(~bad | ~stable), (l1[bad & stable], allow[bad & stable], np.flatnonzero(bad & stable))
    assert (~stable).sum() <= 0.03 * len(ics), (~stable).sum()


def _allowance(orc, pot, omega, dt, S, ics, grid, suspects, per_event):
    allow = np.zeros(len(ics))
    idx = np.flatnonzero(suspects)
    if len(idx):
        allow[idx] = per_event * guard_events(orc, pot, omega, dt, S, ics[idx], grid, 2e-4)
    return allow


def _stable_columns(orc, pot, omega, dt, S, ics, grid, Uo, suspects, gh_v0s=None):
    """True for orbits whose oracle column moves by < 2e-4 (L1) when the
    initial conditions change by 1e-7 relative (checked for the suspects only;
    every other orbit already meets the gate)."""
    stable = np.ones(len(ics), dtype=bool)
    idx = np.flatnonzero(suspects)
    if len(idx):
        U2, _, _ = orc.build_matrix(orc.make_pot(pot), omega, dt, S, ics[idx] * (1 + 1e-7), orc.make_obs(grid),
                                    gh_v0s=gh_v0s)
        stable[idx] = np.abs(U2 - Uo[idx]).sum(axis=1) < 2e-4
    return stable


def test_gh_rows(sw, orc):
    pot, omega = BARRED, 40.0
    grid = _grid(W2, nx=12, ny=10, nR=6, nphi=8, nz=4, gh=1)
    npix = 120
    rng = np.random.default_rng(5)
    v0s = np.stack([rng.normal(0, 40, npix), rng.uniform(60, 160, npix)], 1)
    ics = inputs.disc_ics(inputs.DISC_HALO, 300, seed=105)
    S, dt = 200, inputs.DT_HALF_MYR
    Uo, _, _ = orc.build_matrix(orc.make_pot(pot), omega, dt, S, ics, orc.make_obs(grid), gh_v0s=v0s)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-3)):
        c = ctx_for(sw, prec, pot)
        c.integrate_library(ics, omega, dt, S)
        Ug = c.project(grid, gh_v0s=v0s).copy()
        assert Ug.shape == Uo.shape == (300, 192 + 120 + 480)
        l1 = np.abs(Ug - Uo).sum(axis=1)
        if prec == "fp64":
            assert l1.max() <= tol, (prec, l1.max())
            continue
        allow = _allowance(orc, pot, omega, dt, S, ics, grid, l1 > tol, per_event=18.0 / (4 * S))
        bad = l1 > tol + allow
        stable = _stable_columns(orc, pot, omega, dt, S, ics, grid, Uo, bad, gh_v0s=v0s)
        assert np.all(~bad | ~stable), (l1[bad & stable], allow[bad & stable])
        assert (~stable).sum() <= 0.03 * len(ics)


def test_drift_pass_and_quality_cut(sw, orc):
    """sw_integrate_library's drift pass equals the oracle's Jacobi drift; an
    orbit made non-finite gets status NONFINITE and a zero column."""
    pot, omega = BARRED, 40.0
    ics = inputs.disc_ics(inputs.DISC_HALO, 200, seed=106)
    ics[7, 3] = np.nan
    S, dt = 300, inputs.DT_HALF_MYR
    c = ctx_for(sw, "fp64", pot)
    drift, status = c.integrate_library(ics, omega, dt, S, want_drift=True)
    d_o = orc.drift(orc.make_pot(pot), omega, dt, S, ics)
    ok = np.isfinite(d_o)
    np.testing.assert_allclose(drift[ok], d_o[ok], rtol=1e-6, atol=1e-14)
    assert status[7] == 2 and np.all(status[ok] == (d_o[ok] > 0.1))
    U = c.project(_grid(W2, nx=10, ny=10, nv=8, nR=5, nphi=4, nz=3)).copy()
    assert np.all(U[7] == 0)


def _sampled_drift(orc, po, omega, dt, S, ic, every):
    """The oracle's Jacobi drift max |E_J(t_n) - E_J(0)| / |E_J(0)| over the samples
    n = every, 2 every, ... and the last step."""
    to = orc.trajectory(po, omega, dt, S, ic)
    e0 = orc.jacobi(po, omega, 0.0, to[0])
    ns = sorted(set(range(every, S + 1, every)) | {S})
    return max(abs(orc.jacobi(po, omega, n * dt, to[n]) - e0) / abs(e0) for n in ns)


def test_drift_fp32_against_oracle(sw, orc):
    """The FP32 form's Jacobi drift (Sec. 2.2.2) against the oracle's, orbit by orbit:
    the drift pass of sw_integrate_library checks every step, the projection pass every
    ej_every = 8 steps and the last (its default in FP32), and the oracle's drift is taken
    at the same samples.  Gate: within 3 x the spread of the oracle's own drift under four
    seeded relative perturbations of 1e-6 of the initial condition, plus 1e-6 + 1e-3 of
    the drift; the quality-cut status agrees wherever the drift is not within that band
    of the 0.1 cut."""
    pot, omega = BARRED, 40.0
    po = orc.make_pot(pot)
    ics = inputs.disc_ics(inputs.DISC_HALO, 160, seed=108)
    S, dt = 300, inputs.DT_HALF_MYR
    c = ctx_for(sw, "fp32", pot)
    drift_every, status_every = c.integrate_library(ics, omega, dt, S, want_drift=True)
    c.project(_grid(W2, nx=10, ny=10, nv=8, nR=5, nphi=4, nz=3))
    drift_8, status_8 = c.project_stats(len(ics))
    rng = np.random.default_rng(5100)
    xis = [rng.standard_normal(ics.shape) for _ in range(4)]
    for every, dg, sg in ((1, drift_every, status_every), (8, drift_8, status_8)):
        do = np.array([_sampled_drift(orc, po, omega, dt, S, ic, every) for ic in ics])
        if every == 1:
            np.testing.assert_allclose(do, orc.drift(po, omega, dt, S, ics), rtol=1e-12, atol=1e-15)
        spread = np.zeros(len(ics))
        for xi in xis:
            dp = np.array([_sampled_drift(orc, po, omega, dt, S, ic, every) for ic in ics * (1 + 1e-6 * xi)])
            spread = np.maximum(spread, np.abs(dp - do))
        band = 3 * spread + 1e-6 + 1e-3 * do
        diff = np.abs(dg - do)
        print(f"FP32 drift every {every}: max |diff| {diff.max():.3g}, max diff / band {(diff / band).max():.3g}, "
              f"largest drift {do.max():.3g}")
        assert np.all(diff <= band), (every, np.flatnonzero(diff > band), diff[diff > band], band[diff > band])
        clear = np.abs(do - 0.1) > band
        np.testing.assert_array_equal(sg[clear], (do[clear] > 0.1).astype(np.uint8))


def test_edge_cases(sw, orc):
    c = ctx_for(sw, "fp32", inputs.DISC_HALO)
    with pytest.raises(sw.SwError):
        c.integrate_library(np.zeros((0, 6)), 0.0, 1e-3, 10)
    with pytest.raises(sw.SwError):
        c.integrate_library(np.zeros((2, 6)), 0.0, -1.0, 10)
    c2 = sw.Context(0, "fp32")
    with pytest.raises(sw.SwError):        # no potential yet
        c2.integrate_library(np.ones((2, 6)), 0.0, 1e-3, 10)
    with pytest.raises(sw.SwError):        # project before integrate
        c.project(W1["grid"])
    # orbits that never enter the grid give all-zero columns
    ics = inputs.disc_ics(inputs.DISC_HALO, 5, seed=1)
    ics[:, :3] += np.array([200.0, 0, 0])
    c.integrate_library(ics, 0.0, inputs.DT_HALF_MYR, 20)
    U = c.project(W1["grid"]).copy()
    assert U.shape == (5, 7300) and np.all(U == 0)
    # a single orbit and a single step
    c.integrate_library(inputs.disc_ics(inputs.DISC_HALO, 1, seed=2), 0.0, inputs.DT_HALF_MYR, 1)
    U = c.project(W1["grid"]).copy()
    Uo, _, _ = orc.build_matrix(orc.make_pot(inputs.DISC_HALO), 0.0, inputs.DT_HALF_MYR, 1,
                                inputs.disc_ics(inputs.DISC_HALO, 1, seed=2), orc.make_obs(W1["grid"]))
    np.testing.assert_allclose(U, Uo, atol=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reduce_gh(sw, orc, prec):
    pot, omega = BARRED, 40.0
    grid = _grid(W2, nx=12, ny=10, nv=32, nR=6, nphi=8, nz=4)
    rng = np.random.default_rng(6)
    v0s = np.stack([rng.normal(0, 40, 120), rng.uniform(60, 160, 120)], 1)
    ics = inputs.disc_ics(inputs.DISC_HALO, 260, seed=107)
    c = ctx_for(sw, prec, pot)
    c.integrate_library(ics, omega, inputs.DT_HALF_MYR, 150)
    Uh = c.project(grid)
    Ug = c.reduce_gh(Uh, v0s)
    assert (Ug.M, Ug.N) == (192 + 120 * 5, 260) and Ug.blocks == (192, 120, 480)
    ref = orc.reduce_gh(Uh.copy(), 192, 120, 32, -400.0, 25.0, v0s)   # reduce the GPU's own histogram
    np.testing.assert_allclose(Ug.copy(), ref, rtol=1e-12 if prec == "fp64" else 2e-5,
                               atol=1e-15 if prec == "fp64" else 1e-7)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bundle(sw, orc, prec):
    """sw_bundle against the oracle's bundle mean on the GPU's own matrix, with
    dithered initial conditions (Sec. 2.2.1), a ragged bundle count and the
    n = 1 identity; a size that does not divide N is rejected."""
    pot = BARRED
    base = inputs.disc_ics(inputs.DISC_HALO, 37, seed=111)
    ics = inputs.dither(base, 4, 112, pot)
    assert ics.shape == (148, 6)
    grid = _grid(W2, nx=12, ny=10, nv=8, nR=6, nphi=6, nz=4)
    c = ctx_for(sw, prec, pot)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, 200)
    U = c.project(grid)
    Ug = U.copy()
    B = c.bundle(U, 4)
    assert (B.M, B.N) == (U.M, 37)
    tol = 1e-15 if prec == "fp64" else 3e-7
    np.testing.assert_allclose(B.copy(), orc.bundle(Ug, 4), rtol=tol, atol=0)
    np.testing.assert_array_equal(c.bundle(U, 1).copy(), Ug)
    with pytest.raises(sw.SwError):
        c.bundle(U, 3)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bundled_projection(sw, orc, prec):
    """Bundles accumulated at bin time (option project_bundle): the same means as sw_bundle
    of the unbundled matrix (integer counts, one normalisation), with a realisation cut by
    the quality test (a non-finite initial condition) contributing a zero column to its
    bundle; a bundle size that does not divide the orbit count is rejected."""
    pot = BARRED
    base = inputs.disc_ics(inputs.DISC_HALO, 61, seed=113)
    ics = inputs.dither(base, 4, 114, pot)
    ics[4 * 7 + 2, 3] = np.nan                       # one realisation of bundle 7
    grid = _grid(W2, nx=12, ny=10, nv=8, nR=6, nphi=6, nz=4)
    S = 64
    c = ctx_for(sw, prec, pot)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, S)
    U = c.project(grid)
    ref = c.bundle(U, 4).copy()
    _, status = c.project_stats(len(ics))
    assert status[4 * 7 + 2] == 2
    c.set_option("project_bundle", 4)
    Ub = c.project(grid)
    assert (Ub.M, Ub.N) == (U.M, 61)
    got = Ub.copy()
    np.testing.assert_allclose(got, ref, rtol=3e-7 if prec == "fp32" else 1e-15, atol=0)
    np.testing.assert_array_equal(np.rint(got * 16 * S), np.rint(ref * 16 * S))
    Uo, _, _ = orc.build_matrix(orc.make_pot(pot), 40.0, inputs.DT_HALF_MYR, S, np.nan_to_num(ics), orc.make_obs(grid))
    Uo[4 * 7 + 2] = 0.0
    if prec == "fp64":
        np.testing.assert_allclose(got, orc.bundle(Uo, 4), rtol=0, atol=1e-15)
    c.integrate_library(ics[:-1], 40.0, inputs.DT_HALF_MYR, S)
    with pytest.raises(sw.SwError):
        c.project(grid)
