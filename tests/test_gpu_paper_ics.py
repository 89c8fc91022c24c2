"""The paper's initial conditions (Sec. 2.2.1: double-exponential disc with h_R = 3.5,
h_z = 1.2 kpc and velocities from the Jeans equations in the azimuthally averaged
potential; inputs.paper_ics, pinned on the CPU in tests/test_inputs_paper_ics.py) through
the GPU path: dithered into bundles of four, integrated in the barred potential and
projected with the bundles accumulated at bin time, against the oracle on the same
initial conditions (FP64 counts bit-exact over 64 steps; FP32 counts exact outside the
guard band), and the weight solve on the bundled matrix against the oracle's
Lawson-Hanson on that matrix (chi^2 within 1e-4)."""
from _guard import guard_events
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


@pytest.fixture(scope="module")
def ics():
    base = inputs.paper_ics(BARRED, 150, seed=5101)
    return inputs.dither(base, 4, 5102, BARRED)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_ics_bundled_counts(sw, orc, ics, prec):
    grid = dict(W2["grid"], nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    S = 64
    c = sw.Context(0, prec)
    c.set_potential(BARRED)
    c.set_option("project_bundle", 4)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, S)
    Ub = c.project(grid).copy()
    assert Ub.shape[0] == len(ics) // 4
    Uo, _, so = orc.build_matrix(orc.make_pot(BARRED), 40.0, inputs.DT_HALF_MYR, S, ics, orc.make_obs(grid))
    # per-orbit integer counts of the oracle, summed over each bundle (16 S = 4 copies x S x 4 dithers)
    co = np.rint(Uo * 4 * S).reshape(-1, 4, Uo.shape[1]).sum(1)
    cg = np.rint(Ub * 16 * S)
    if prec == "fp64":
        np.testing.assert_array_equal(cg, co)
    else:
        near = guard_events(orc, BARRED, 40.0, inputs.DT_HALF_MYR, S, ics, grid, 1e-5).reshape(-1, 4).sum(1)
        diff = np.abs(cg - co).sum(1)
        assert np.all(diff <= 2 * near), (np.flatnonzero(diff > 2 * near), diff[diff > 2 * near])


def test_paper_ics_solve(sw, orc, ics):
    grid = dict(W2["grid"], nx=16, ny=16, nv=12, nR=8, nphi=8, nz=4)
    c = sw.Context(0, "fp32")
    c.set_potential(BARRED)
    c.set_option("project_bundle", 4)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, 400)
    U = c.project(grid)
    rows = U.copy().T.copy()
    blocks = inputs.row_blocks(grid)
    y0 = rows @ inputs.true_weights(U.N, 5103)
    sig = inputs.mock_sigma(y0, blocks)
    y = y0 + sig * inputs.noise(len(y0), 5104)
    w, chi2 = c.solve_weights(U, y, sig, 1.0)
    Ut, yt = orc.whiten(rows, y, sig)
    H, q = orc.normal_equations(Ut, yt, 1.0)
    w_o = orc.nnls_lh_normal(H, q)
    chi2_o = orc.chi2_parts(rows, y, sig, w_o, 1.0, blocks["dens"][1])
    assert np.all(w >= 0)
    np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=1e-4)
