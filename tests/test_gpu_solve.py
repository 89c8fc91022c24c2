"""GPU parity of the weight solve (Sec. 2.3-2.4) through the C-ABI.

Solve parity is decoupled from matrix parity: the GPU solves on its own orbit
matrix, the oracle (Lawson-Hanson on the normal equations, FP64) solves on the
same matrix exported from the GPU; chi^2 must agree within 1e-4 relative.
Both Gram spaces are covered (orbit space N <= M and constraint space M < N),
with lambda = 1 and lambda = 0.  At the full axisym_2k size the GPU solution
is checked by its FP64 KKT certificate.
"""
import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

pytestmark = pytest.mark.gpu
W1 = inputs.WORKLOADS["axisym_2k"]
BARRED = dict(inputs.DISC_HALO, **inputs.BAR)


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    return swmod


def _mock(orc, U_rows, blocks, seed_w=2001, seed_n=2002, gh_err=None):
    """Mock data from the given matrix (item: w_true ~ U(0,2), 2% errors)."""
    N = U_rows.shape[1]
    w_true = inputs.true_weights(N, seed_w)
    y0 = U_rows @ w_true
    sig = inputs.mock_sigma(y0, blocks, gh_err=gh_err)
    y = y0 + sig * inputs.noise(len(y0), seed_n)
    return y, sig


def _oracle_solve(orc, U_rows, y, sig, lam, n_dens):
    Ut, yt = orc.whiten(U_rows, y, sig)
    H, q = orc.normal_equations(Ut, yt, lam)
    w = orc.nnls_lh_normal(H, q)
    return w, orc.chi2_parts(U_rows, y, sig, w, lam, n_dens), H, q


def _build(sw, prec, pot, omega, ics, S, grid, gh_v0s=None):
    c = sw.Context(0, prec)
    c.set_potential(pot)
    c.integrate_library(ics, omega, inputs.DT_HALF_MYR, S)
    U = c.project(grid, gh_v0s=gh_v0s)
    return c, U


@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("lam", [1.0, 0.0])
def test_solve_orbit_space(sw, orc, prec, lam, solver):
    """solver 0: the default choice (active set here); 2: the paper's ADMM with refinement and polish."""
    ics = inputs.disc_ics(W1["potential"], 500, seed=201)
    c, U = _build(sw, prec, W1["potential"], 0.0, ics, 1000, W1["grid"])
    c.set_option("solver", solver)
    Ug = U.copy().T.copy()                       # (M, N)
    blocks = inputs.row_blocks(W1["grid"])
    y, sig = _mock(orc, Ug, blocks)
    w, chi2 = c.solve_weights(U, y, sig, lam)
    info = c.solve_info()
    assert not info["constraint_space"]
    w_o, chi2_o, H, q = _oracle_solve(orc, Ug, y, sig, lam, blocks["dens"][1])
    assert np.all(w >= 0)
    np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=1e-4)
    np.testing.assert_allclose(chi2[2], chi2_o[2], rtol=1e-3, atol=1e-9 * max(1.0, chi2_o[0]))


@pytest.mark.parametrize("solver", [0, 2])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("lam", [1.0, 0.0])
def test_solve_constraint_space_gh(sw, orc, prec, lam, solver):
    """M < N with GH rows: the default choice (active set for lambda > 0, ADMM for lambda = 0) and
    the paper's ADMM throughout."""
    grid = dict(W1["grid"], nx=6, ny=6, nR=5, nphi=4, nz=3, gh=1, incl=0.9)
    npix = 36
    ics = inputs.disc_ics(BARRED, 700, seed=202)
    po = orc.make_pot(BARRED)
    mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 500, ics, orc.make_obs(grid), np.ones(len(ics)))
    v0s, gh_err = inputs.gh_reference(mom)
    c, U = _build(sw, prec, BARRED, 40.0, ics, 500, grid, gh_v0s=v0s)
    c.set_option("solver", solver)
    assert U.M == 60 + 36 + 144 and U.N == 700
    Ug = U.copy().T.copy()
    blocks = inputs.row_blocks(grid)
    y, sig = _mock(orc, Ug, blocks, gh_err=gh_err)
    w, chi2 = c.solve_weights(U, y, sig, lam)
    assert c.solve_info()["constraint_space"]
    w_o, chi2_o, H, q = _oracle_solve(orc, Ug, y, sig, lam, blocks["dens"][1])
    assert np.all(w >= 0)
    np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=1e-4)


def test_solve_full_axisym_kkt_certificate(sw, orc):
    """axisym_2k at full size: the returned weights satisfy the FP64 KKT
    conditions of the exact problem on the exported matrix."""
    W = W1
    ics = inputs.disc_ics(W["potential"], W["n_orb"], seed=W["seeds"]["ic"])
    c, U = _build(sw, "fp32", W["potential"], 0.0, ics, W["nsteps"], W["grid"])
    Ug = U.copy().T.copy()
    blocks = inputs.row_blocks(W["grid"])
    y, sig = _mock(orc, Ug, blocks)
    w, chi2 = c.solve_weights(U, y, sig, W["lam"])
    Ut, yt = orc.whiten(Ug, y, sig)
    H, q = orc.normal_equations(Ut, yt, W["lam"])
    k = orc.kkt_residual(H, q, w)
    assert k["neg_w"] == 0.0
    assert k["pg_inf"] <= 1e-6 * np.abs(q).max(), k
    # chi2 parts recomputed in FP64 on the host
    np.testing.assert_allclose(chi2, orc.chi2_parts(Ug, y, sig, w, W["lam"], blocks["dens"][1]), rtol=1e-9)
    # the certificate bounds the objective gap: f(w) - f* <= ||P(g)||^2 / (2 mu)
    gap_bound = k["pg_norm2"] / (2 * 2 * W["lam"] / len(w))
    assert gap_bound <= 1e-4 * chi2[0]


def test_solve_rejects_bad_errors(sw, orc):
    ics = inputs.disc_ics(W1["potential"], 50, seed=203)
    c, U = _build(sw, "fp32", W1["potential"], 0.0, ics, 50, W1["grid"])
    y = np.ones(U.M); s = np.ones(U.M); s[3] = 0.0
    with pytest.raises(sw.SwError):
        c.solve_weights(U, y, s, 1.0)
    with pytest.raises(sw.SwError):
        c.solve_weights(U, y, np.ones(U.M), -1.0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_solve_active_set_path(sw, orc, prec):
    """The active-set path (used above 8 192 orbits) forced on a small problem
    with more orbits than constraints: exact chi^2 (1e-4 relative to the
    oracle's Lawson-Hanson) and its KKT certificate met."""
    grid = dict(W1["grid"], nx=6, ny=6, nR=5, nphi=4, nz=3, gh=1, incl=0.9)
    ics = inputs.disc_ics(BARRED, 700, seed=202)
    po = orc.make_pot(BARRED)
    mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 500, ics, orc.make_obs(grid), np.ones(len(ics)))
    v0s, gh_err = inputs.gh_reference(mom)
    c, U = _build(sw, prec, BARRED, 40.0, ics, 500, grid, gh_v0s=v0s)
    c.set_option("orbit_direct_max", 0)
    Ug = U.copy().T.copy()
    blocks = inputs.row_blocks(grid)
    y, sig = _mock(orc, Ug, blocks, gh_err=gh_err)
    w, chi2 = c.solve_weights(U, y, sig, 1.0)
    info = c.solve_info()
    assert info["kkt_met"] and info["ws_size"] == int((w > 0).sum())
    w_o, chi2_o, H, q = _oracle_solve(orc, Ug, y, sig, 1.0, blocks["dens"][1])
    assert np.all(w >= 0)
    np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=1e-4)
    k = orc.kkt_residual(H, q, w)
    assert k["pg_inf"] <= 1e-6 * np.abs(q).max(), k


def test_cooperative_factorisation_matches_per_step_launches(sw, orc):
    """The one-launch Cholesky + inverse (cooperative grid) and the per-step
    launches give the same active-set solution."""
    grid = dict(W1["grid"], nx=8, ny=8, nR=5, nphi=4, nz=3, gh=1, incl=0.9)
    ics = inputs.disc_ics(BARRED, 1500, seed=205)
    po = orc.make_pot(BARRED)
    mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 300, ics, orc.make_obs(grid), np.ones(len(ics)))
    v0s, gh_err = inputs.gh_reference(mom)
    out = []
    for coop in (0, 1):
        c, U = _build(sw, "fp32", BARRED, 40.0, ics, 300, grid, gh_v0s=v0s)
        c.set_option("orbit_direct_max", 0)
        c.set_option("chol_coop", coop)
        Ug = U.copy().T.copy()
        y, sig = _mock(orc, Ug, inputs.row_blocks(grid), gh_err=gh_err)
        w, chi2 = c.solve_weights(U, y, sig, 1.0)
        assert c.solve_info()["kkt_met"]
        out.append((w, chi2))
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-7)
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-4, atol=1e-6 * out[0][0].max())


def test_factor_bordering_matches_refactoring(sw, orc):
    """Pivoting steps that add a few orbits to the factored set extend its factor by bordering
    (option as_border) and mask the orbits that left it (as_mask) instead of refactoring: the
    same solution as refactoring at every step, with fewer factorisations and about as many
    conjugate-gradient steps (the preconditioner is corrected to the exact inverse on the passive
    set), both meeting the KKT certificate, and the oracle's chi^2."""
    grid = dict(W1["grid"], nx=8, ny=8, nR=5, nphi=4, nz=3, gh=1, incl=0.9)
    ics = inputs.disc_ics(BARRED, 1500, seed=205)
    po = orc.make_pot(BARRED)
    mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 300, ics, orc.make_obs(grid), np.ones(len(ics)))
    v0s, gh_err = inputs.gh_reference(mom)
    out = []
    for border, mask in ((0, 0.0), (256, 0.1)):
        c, U = _build(sw, "fp32", BARRED, 40.0, ics, 300, grid, gh_v0s=v0s)
        c.set_option("orbit_direct_max", 0)
        c.set_option("as_block", 16)
        c.set_option("as_border", border)
        c.set_option("as_mask", mask)
        Ug = U.copy().T.copy()
        blocks = inputs.row_blocks(grid)
        y, sig = _mock(orc, Ug, blocks, gh_err=gh_err)
        c.reset_stats()
        w, chi2 = c.solve_weights(U, y, sig, 1.0)
        info = c.solve_info()
        assert info["kkt_met"]
        borders = c.kernel_stats().get("factor_border", {}).get("launches", 0)
        out.append((w, chi2, borders, info["refine_rounds"], info["admm_iterations"]))
    print(f"factorisations {out[0][3]}, CG steps {out[0][4]} (refactoring) against {out[1][3]}, {out[1][4]} "
          f"(bordering, {out[1][2]} border launches)")
    assert out[0][2] == 0 and out[1][2] > 0
    assert out[1][3] < out[0][3]
    assert out[1][4] <= 1.5 * out[0][4] + 10
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-7)
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-4, atol=1e-6 * out[0][0].max())
    w_o, chi2_o, H, q = _oracle_solve(orc, Ug, y, sig, 1.0, blocks["dens"][1])
    np.testing.assert_allclose(out[1][1][:2], chi2_o[:2], rtol=1e-4)


def test_solve_working_set_path(sw, orc):
    """The ADMM working-set option for very many orbits on a small problem with
    the direct path disabled: its chi^2 approaches the exact one and its
    weights satisfy the KKT conditions to the solver's reported level."""
    grid = dict(W1["grid"], nx=6, ny=6, nR=5, nphi=4, nz=3, gh=1, incl=0.9)
    ics = inputs.disc_ics(BARRED, 700, seed=202)
    po = orc.make_pot(BARRED)
    mom = orc.pixel_moments(po, 40.0, inputs.DT_HALF_MYR, 500, ics, orc.make_obs(grid), np.ones(len(ics)))
    v0s, gh_err = inputs.gh_reference(mom)
    c, U = _build(sw, "fp32", BARRED, 40.0, ics, 500, grid, gh_v0s=v0s)
    c.set_option("orbit_direct_max", 0)
    c.set_option("large_solver", 1)
    c.set_option("ws_rounds", 12)
    Ug = U.copy().T.copy()
    blocks = inputs.row_blocks(grid)
    y, sig = _mock(orc, Ug, blocks, gh_err=gh_err)
    w, chi2 = c.solve_weights(U, y, sig, 1.0, allow_nonconv=True)
    info = c.solve_info()
    assert info["ws_rounds"] >= 1 and info["ws_size"] > 0
    w_o, chi2_o, H, q = _oracle_solve(orc, Ug, y, sig, 1.0, blocks["dens"][1])
    assert np.all(w >= 0)
    np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=2e-3)
