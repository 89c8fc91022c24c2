"""Batched model construction (one persistent launch over many trial
potentials with uneven orbit counts, autotuned and replayed from a CUDA graph):
every model's matrix and chi^2 against the FP64 oracle, and the batch against
the single-model path on the same inputs."""
from _guard import guard_events
import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    return swmod


def _models(n, seed):
    th = inputs.draw_box(n, seed)
    return [inputs.box_model(t) for t in th]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("gh", [0, 1])
def test_batch_against_oracle(sw, orc, prec, gh):
    """Each model of one batched launch against the oracle's build_matrix of that model
    (its own potential, pattern speed and viewing angles): FP64 bin counts bit-exact over
    64 steps and GH rows to 1e-12; FP32 counts exact outside the 1e-5 bin-width guard band
    and GH rows within L1 2e-3 plus the guard-band allowance.  Then each model's chi^2
    from a solve on the batch's own matrix against the oracle's Lawson-Hanson on the same
    (exported) matrix, within 1e-4 relative."""
    grid = dict(inputs.WORKLOADS["batched_64"]["grid"], nx=10, ny=8, nR=5, nphi=6, nz=3, nv=12, gh=gh)
    models = _models(3, 3101 + gh)
    counts = np.array([260, 389, 130])          # uneven, several 64/128-orbit tiles and ragged tails
    S, dt = 64, inputs.DT_HALF_MYR
    ics = [inputs.disc_ics(m["potential"], n, seed=720 + k) for k, (m, n) in enumerate(zip(models, counts))]
    npix = grid["nx"] * grid["ny"]
    blocks = inputs.row_blocks(grid)
    nc = blocks["pix"][1]
    c = sw.Context(0, prec)
    gk = [dict(grid, incl=m["incl"], bar_angle=m["bar_angle"]) for m in models]
    v0s, errs = [], []
    for k, m in enumerate(models):
        if gh:   # per-pixel GH reference from each model's own LOSVD (oracle moments)
            mom = orc.pixel_moments(orc.make_pot(m["potential"]), m["omega_p"], dt, S, ics[k],
                                    orc.make_obs(dict(gk[k], gh=0)), np.ones(counts[k]))
            v, e = inputs.gh_reference(mom)
            v0s.append(v); errs.append(e)
        else:
            v0s.append(None); errs.append(None)
    b = sw.Batch(c, counts, S, grid)
    b.set_models([m["potential"] for m in models], [m["omega_p"] for m in models],
                 [[m["incl"], 0.0, m["bar_angle"]] for m in models], dt, np.concatenate(ics),
                 np.stack(v0s) if gh else None)
    b.run()
    drift_b, status_b = b.stats()
    off = np.concatenate([[0], np.cumsum(counts)])
    for k, m in enumerate(models):
        Uo, drift_o, status_o = orc.build_matrix(orc.make_pot(m["potential"]), m["omega_p"], dt, S, ics[k],
                                                 orc.make_obs(gk[k]), gh_v0s=v0s[k])
        Ub = b.matrix(k).copy()
        assert Ub.shape == Uo.shape
        cb, co = np.rint(Ub[:, :nc] * 4 * S), np.rint(Uo[:, :nc] * 4 * S)
        if not gh:
            cb = np.concatenate([cb, np.rint(Ub[:, nc:] * 4 * S)], 1)
            co = np.concatenate([co, np.rint(Uo[:, nc:] * 4 * S)], 1)
        np.testing.assert_array_equal(status_b[off[k]:off[k + 1]], status_o)
        if prec == "fp64":
            np.testing.assert_array_equal(cb, co)
            np.testing.assert_allclose(Ub, Uo, rtol=0, atol=1e-12 * max(1.0, np.abs(Uo).max()))
            np.testing.assert_allclose(drift_b[off[k]:off[k + 1]], drift_o, rtol=1e-6, atol=1e-13)
        else:
            near = guard_events(orc, m["potential"], m["omega_p"], dt, S, ics[k], gk[k], 1e-5)
            diff = np.abs(cb - co).sum(axis=1)
            assert np.all(diff <= 2 * near), (k, np.flatnonzero(diff > 2 * near))
            if gh:
                l1 = np.abs(Ub[:, nc:] - Uo[:, nc:]).sum(axis=1)
                allow = 18.0 / (4 * S) * guard_events(orc, m["potential"], m["omega_p"], dt, S, ics[k], gk[k],
                                                      2e-4)
                assert np.all(l1 <= 2e-3 + allow), (k, l1.max())
        # chi^2 of the batch's matrix: GPU solve vs the oracle's Lawson-Hanson on that matrix
        rows = Ub.T.copy()
        w_true = inputs.true_weights(counts[k], 3200 + k)
        y0 = rows @ w_true
        sig = inputs.mock_sigma(y0, blocks, gh_err=errs[k])
        y = y0 + sig * inputs.noise(len(y0), 3300 + k)
        w, chi2 = c.solve_weights(b.matrix(k), y, sig, 1.0)
        Ut, yt = orc.whiten(rows, y, sig)
        H, q = orc.normal_equations(Ut, yt, 1.0)
        w_o = orc.nnls_lh_normal(H, q)
        chi2_o = orc.chi2_parts(rows, y, sig, w_o, 1.0, blocks["dens"][1])
        assert np.all(w >= 0)
        np.testing.assert_allclose(chi2[:2], chi2_o[:2], rtol=1e-4)
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("gh", [0, 1])
def test_batch_matches_single_model_path(sw, prec, gh):
    grid = dict(inputs.WORKLOADS["batched_64"]["grid"], nx=10, ny=8, nR=5, nphi=6, nz=3, nv=12, gh=gh)
    models = _models(3, 3001 + gh)
    counts = np.array([300, 517, 130])
    S, dt = 120, inputs.DT_HALF_MYR
    ics = [inputs.disc_ics(m["potential"], n, seed=700 + k) for k, (m, n) in enumerate(zip(models, counts))]
    npix = grid["nx"] * grid["ny"]
    rng = np.random.default_rng(5)
    v0s = [np.stack([rng.normal(0, 30, npix), rng.uniform(60, 160, npix)], 1) for _ in models]
    c = sw.Context(0, prec)
    b = sw.Batch(c, counts, S, grid)
    b.set_models([m["potential"] for m in models], [m["omega_p"] for m in models],
                 [[m["incl"], 0.0, m["bar_angle"]] for m in models], dt, np.concatenate(ics),
                 np.stack(v0s) if gh else None)
    b.run()
    info = b.info()
    assert info["autotuned"] and info["graph"] and info["threads"] in (64, 128, 256)
    assert sum(t > 0 for t in info["probe_ms"]) == 12
    first = [b.matrix(k).copy() for k in range(3)]
    drift_b, status_b = b.stats()
    b.run()                                   # graph replay
    for k in range(3):
        np.testing.assert_array_equal(b.matrix(k).copy(), first[k])
    off = np.concatenate([[0], np.cumsum(counts)])
    for k, m in enumerate(models):
        c1 = sw.Context(0, prec)
        c1.set_potential(m["potential"])
        c1.integrate_library(ics[k], m["omega_p"], dt, S)
        U = c1.project(dict(grid, incl=m["incl"], bar_angle=m["bar_angle"]), gh_v0s=v0s[k] if gh else None)
        Us = U.copy()
        nc = U.blocks[0] + U.blocks[1]              # count rows (density, pixel mass): exact
        np.testing.assert_array_equal(first[k][:, :nc], Us[:, :nc])
        if gh:   # GH sums: the two kernels may contract the FP32 GH arithmetic differently
            np.testing.assert_allclose(first[k][:, nc:], Us[:, nc:], rtol=0,
                                       atol=(1e-6 if prec == "fp32" else 1e-14) * np.abs(Us).max())
        else:
            np.testing.assert_array_equal(first[k], Us)
        d1, s1 = c1.project_stats(counts[k])
        np.testing.assert_array_equal(status_b[off[k]:off[k + 1]], s1)
        np.testing.assert_allclose(drift_b[off[k]:off[k + 1]], d1, rtol=0, atol=0)
        U.free()
    # a view is solved like any matrix and cannot be freed by the caller
    V = b.matrix(1)
    y = V.apply(inputs.true_weights(V.N, 11))
    sig = 0.02 * np.maximum(np.abs(y), 1e-3 * np.abs(y).max() + 1e-12)
    w, chi2 = c.solve_weights(V, y, sig, 1.0, allow_nonconv=True)
    assert np.all(w >= 0) and np.isfinite(chi2).all()
    assert sw.lib().sw_matrix_free(V.handle) != sw.SW_OK
    b.close()
