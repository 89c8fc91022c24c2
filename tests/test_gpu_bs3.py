"""The paper's own integrator on the GPU: the adaptive Bogacki-Shampine 3(2) pair in
the frame rotating with the bar (Sec. 2.2.2), a fixed number of accepted steps per
orbit and samples weighted by their step over the orbit's total time (Sec. 2.2.4),
selected by the option integrator = 1, against the oracle's build_matrix_bs3 on the
same seeded inputs, through the C-ABI.

FP64: per-orbit L1 difference of the columns <= 1e-6 (the two sides take the same
step sequence; their step sizes differ by rounding only), identical status, drift
to 1e-9.  FP32: the step controller's decisions depend on the working precision, so
an orbit's FP32 step sequence can leave the FP64 one; each column is held to the
oracle's own spread under perturbations of the initial condition, and most columns
meet the plain per-orbit L1 gate of 1e-3 outright.  An orbit abandoned before its first
accepted step keeps an all-zero column."""
import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

pytestmark = pytest.mark.gpu

BARRED = dict(inputs.DISC_HALO, **inputs.BAR)
W2 = inputs.WORKLOADS["barred_100k"]


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    return swmod


def _grid(**kw):
    g = dict(W2["grid"], nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    g.update(kw)
    return g


def _gpu(sw, prec, ics, S, grid, gh_v0s=None):
    c = sw.Context(0, prec)
    c.set_potential(BARRED)
    c.set_option("integrator", 1)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, S)
    U = c.project(grid, gh_v0s=gh_v0s).copy()
    drift, status = c.project_stats(len(ics))
    return U, drift, status


@pytest.mark.parametrize("gh", [0, 1])
def test_bs3_fp64_columns(sw, orc, gh):
    ics = inputs.disc_ics(inputs.DISC_HALO, 300, seed=120)   # two 128-orbit CTAs and a ragged tail
    S = 300
    v0s = None
    grid = _grid(gh=gh)
    if gh:
        rng = np.random.default_rng(121)
        v0s = np.stack([rng.normal(0, 40, 400), rng.uniform(60, 160, 400)], 1)
    Uo, drift_o, status_o = orc.build_matrix_bs3(orc.make_pot(BARRED), 40.0, orc.bs3_opts(), S, ics,
                                                 orc.make_obs(grid), gh_v0s=v0s)
    Ug, drift_g, status_g = _gpu(sw, "fp64", ics, S, grid, v0s)
    assert Ug.shape == Uo.shape
    np.testing.assert_array_equal(status_g, status_o)
    l1 = np.abs(Ug - Uo).sum(axis=1)
    print(f"BS3 FP64 (gh={gh}): per-orbit L1 max {l1.max():.3g}, median {np.median(l1):.3g}")
    assert l1.max() <= 1e-6, (np.argmax(l1), l1.max())
    ok = status_o == 0
    np.testing.assert_allclose(drift_g[ok], drift_o[ok], rtol=0, atol=1e-9)
    # every kept column holds the orbit's unit mass in the density block (samples inside the grid)
    nd = grid["nR"] * grid["nphi"] * grid["nz"]
    assert np.all(Ug[ok, :nd].sum(1) <= 1.0 + 1e-12)


def test_bs3_abandoned_orbit_has_zero_column(sw, orc):
    """A non-finite initial condition ends the orbit before its first accepted step
    (t_total = 0): its column stays all zero, with no division by the zero time."""
    ics = inputs.disc_ics(inputs.DISC_HALO, 40, seed=122)
    ics[5, 4] = np.nan
    for prec in ("fp64", "fp32"):
        Ug, drift, status = _gpu(sw, prec, ics, 50, _grid())
        assert status[5] == 2
        assert np.all(Ug[5] == 0.0)
        assert np.all(np.isfinite(Ug))
        assert np.all(status[np.arange(40) != 5] != 2)


def test_bs3_fp32_columns(sw, orc):
    """FP32 form against the FP64 oracle.  The controller accepts or rejects a trial step by
    comparing an error estimate -- a small difference of stage derivatives -- with the
    tolerance in the working precision, so an FP32 step sequence can part from the FP64 one
    and an orbit's samples then fall at other (equally valid) times.  Gate: each column's L1
    difference at most 3 x the oracle's own spread plus 1e-3, the spread being the largest L1
    change of the oracle's column under four seeded relative perturbations of 3e-5 of the
    initial condition (the full-size reading of the fixed-step path) or under a relative
    change of 1e-3 of the tolerance (another accept/reject sequence); the median difference at
    most the median initial-condition spread; nine columns in ten within the plain 1e-3
    matrix gate."""
    ics = inputs.disc_ics(inputs.DISC_HALO, 300, seed=120)
    S = 300
    grid = _grid()
    po, obs, opts = orc.make_pot(BARRED), orc.make_obs(grid), orc.bs3_opts()
    Uo, _, status_o = orc.build_matrix_bs3(po, 40.0, opts, S, ics, obs)
    Ug, _, status_g = _gpu(sw, "fp32", ics, S, grid)
    np.testing.assert_array_equal(status_g, status_o)
    spread = np.zeros(len(ics))
    for k in range(4):
        xi = np.random.default_rng(9100 + k).standard_normal(ics.shape)
        Up, _, _ = orc.build_matrix_bs3(po, 40.0, opts, S, ics + 3e-5 * np.abs(ics) * xi, obs)
        spread = np.maximum(spread, np.abs(Up - Uo).sum(axis=1))
    spread_tol = np.zeros(len(ics))
    for fac in (1.0 + 1e-3, 1.0 - 1e-3):
        Up, _, _ = orc.build_matrix_bs3(po, 40.0, orc.bs3_opts(rtol=1e-4 * fac), S, ics, obs)
        spread_tol = np.maximum(spread_tol, np.abs(Up - Uo).sum(axis=1))
    l1 = np.abs(Ug - Uo).sum(axis=1)
    print(f"BS3 FP32: per-orbit L1 median {np.median(l1):.3g}, max {l1.max():.3g}; "
          f"{(l1 <= 1e-3).mean():.3f} of columns within 1e-3; median spread {np.median(spread):.3g} "
          f"(initial condition), {np.median(spread_tol):.3g} (tolerance)")
    bad = l1 > 3.0 * np.maximum(spread, spread_tol) + 1e-3
    assert not bad.any(), (np.flatnonzero(bad), l1[bad], spread[bad])
    assert np.median(l1) <= np.median(spread)
    assert (l1 <= 1e-3).mean() >= 0.9
