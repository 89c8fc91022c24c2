"""Bootstrap solves and the marginalised chi^2 (Sec. 2.4 and the model-likelihood passage
after it) through sw_solve_bootstrap, against the oracle's bootstrap_solve / chi2_model on
the GPU's own matrix (decoupled parity: the oracle solves every realisation by
Lawson-Hanson on the exported matrix with the same draws).  Gates: every chi2_b and
chi2_model within 1e-4 relative, every weight set non-negative and within the KKT
conditions of its realisation's problem."""
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


def _problem(sw, orc, prec, n_orb, seed, gh=True):
    grid = dict(W2["grid"], nx=10, ny=10, nv=16, nR=6, nphi=6, nz=4, gh=int(gh))
    ics = inputs.disc_ics(inputs.DISC_HALO, n_orb, seed=seed)
    po = orc.make_pot(BARRED)
    v0s, gh_err = None, None
    if gh:
        mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 300, ics, orc.make_obs(dict(grid, gh=0)),
                                np.ones(n_orb))
        v0s, gh_err = inputs.gh_reference(mom)
    c = sw.Context(0, prec)
    c.set_potential(BARRED)
    c.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, 300)
    U = c.project(grid, gh_v0s=v0s)
    rows = U.copy().T.copy()
    blocks = inputs.row_blocks(grid)
    y0 = rows @ inputs.true_weights(n_orb, seed + 1)
    sig = inputs.mock_sigma(y0, blocks, gh_err=gh_err)
    y = y0 + sig * inputs.noise(len(y0), seed + 2)
    return c, U, rows, y, sig, blocks["dens"][1]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bootstrap_against_oracle(sw, orc, prec):
    B, lam = 16, 1.0
    c, U, rows, y, sig, nd = _problem(sw, orc, prec, 320, 4100)
    xi = inputs.bootstrap_noise(U.M, B, 4200)
    w, chi_b, chi_m = c.solve_bootstrap(U, y, sig, lam, xi, want_weights=True)
    W_o, chi_o, cm_o = orc.bootstrap_solve(rows, y, sig, lam, nd, xi)
    assert w.shape == (B, U.N) and np.all(w >= 0) and np.all(np.isfinite(chi_b))
    print(f"bootstrap ({prec}): chi2_b rel. diff max {np.max(np.abs(chi_b - chi_o) / chi_o):.3g}, "
          f"chi2_model {chi_m:.6g} vs {cm_o:.6g}; spread of chi2_b {chi_o.std():.3g}")
    np.testing.assert_allclose(chi_b, chi_o, rtol=1e-4)
    assert abs(chi_m - cm_o) <= 1e-4 * cm_o
    # each weight set is the exact minimiser of its own realisation's problem (KKT in FP64)
    Yb = orc.bootstrap_data(y, sig, nd, xi)
    Ut = rows / sig[:, None]
    H = Ut.T @ Ut + (2.0 * lam / U.N) * np.eye(U.N)
    for b in range(B):
        k = orc.kkt_residual(H, Ut.T @ (Yb[b] / sig), w[b])
        assert k["pg_inf"] <= 1e-6 * np.abs(Ut.T @ (Yb[b] / sig)).max(), (b, k)
    # the realisations differ: the bootstrap is not a copy of one solve
    assert chi_o.std() > 0 and np.abs(w[0] - w[1]).max() > 0


def test_bootstrap_edge_cases(sw, orc):
    c, U, rows, y, sig, nd = _problem(sw, orc, "fp32", 200, 4300, gh=False)
    # one realisation with zero draws: the plain solve, and chi2_model = chi2_b
    xi = np.zeros((1, U.M))
    _, chi_b, chi_m = c.solve_bootstrap(U, y, sig, 1.0, xi)
    w0, chi = c.solve_weights(U, y, sig, 1.0)
    assert chi_m == pytest.approx(chi_b[0], rel=1e-15)
    assert chi_b[0] == pytest.approx(chi[1], rel=1e-9)
    with pytest.raises(sw.SwError):
        c.solve_bootstrap(U, y, sig, 1.0, np.zeros((0, U.M)))
    if U.N > U.M:
        with pytest.raises(sw.SwError):
            c.solve_bootstrap(U, y, sig, 0.0, np.zeros((2, U.M)))
