"""Pins for the oracle's bootstrap solves and the marginalised chi^2 (Sec. 2.4-2.5):
B realisations of the observed rows perturbed by their errors (the 3-D density rows
are not bootstrapped), one NNLS per realisation with the shared matrix, and
chi2_model = -2 ln of the bootstrap-averaged likelihood exp(-chi2_b / 2).

Closed forms: a single or repeated chi2_b returns itself; adding a constant to every
chi2_b adds it to chi2_model; two values d apart give chi2_min - 2 ln((1 + e^{-d/2})/2);
one value far below the rest gives chi2_min + 2 ln B; values near 1e6 neither
overflow nor underflow.  Invariants: zero draws reproduce the single solve; every
bootstrap weight set meets its own KKT conditions.
"""
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs


def test_chi2_model_closed_forms(orc):
    assert orc.chi2_model([123.4]) == pytest.approx(123.4, rel=1e-15)
    assert orc.chi2_model([77.0] * 100) == pytest.approx(77.0, rel=1e-15)
    c = np.array([10.0, 13.5, 11.2, 19.0])
    assert orc.chi2_model(c + 1000.0) == pytest.approx(orc.chi2_model(c) + 1000.0, rel=1e-13)
    d = 3.7
    assert orc.chi2_model([50.0, 50.0 + d]) == pytest.approx(50.0 - 2 * math.log((1 + math.exp(-d / 2)) / 2),
                                                              rel=1e-14)
    B = 100
    far = np.full(B, 5e6)
    far[17] = 1e6
    assert orc.chi2_model(far) == pytest.approx(1e6 + 2 * math.log(B), rel=1e-14)
    big = 1e6 + np.arange(100, dtype=float)
    v = orc.chi2_model(big)
    assert math.isfinite(v) and big.min() <= v <= big.min() + 2 * math.log(100)


def test_bootstrap_data_perturbs_observed_rows_only(orc):
    rng = np.random.default_rng(3)
    M, nd, B = 40, 12, 500
    y = rng.uniform(1, 5, M)
    sig = rng.uniform(0.1, 0.3, M)
    xi = inputs.bootstrap_noise(M, B, 11)
    Y = orc.bootstrap_data(y, sig, nd, xi)
    assert Y.shape == (B, M)
    np.testing.assert_array_equal(Y[:, :nd], np.repeat(y[None, :nd], B, 0))
    np.testing.assert_allclose((Y[:, nd:] - y[nd:]) / sig[nd:], xi[:, nd:], rtol=1e-12, atol=1e-12)
    z = ((Y[:, nd:] - y[nd:]) / sig[nd:]).ravel()
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05


def _problem(seed=5, M=36, N=10, nd=8):
    rng = np.random.default_rng(seed)
    U = rng.uniform(0, 1, (M, N)) ** 3
    w = rng.uniform(0, 2, N)
    y0 = U @ w
    sig = 0.05 * y0 + 0.01
    y = y0 + sig * rng.standard_normal(M)
    return U, y, sig, nd


def test_zero_draws_reproduce_the_single_solve(orc):
    U, y, sig, nd = _problem()
    lam = 1.0
    W, chi, cm = orc.bootstrap_solve(U, y, sig, lam, nd, np.zeros((4, len(y))))
    Ut, yt = orc.whiten(U, y, sig)
    H, q = orc.normal_equations(Ut, yt, lam)
    w1 = orc.nnls_lh_normal(H, q)
    for b in range(4):
        np.testing.assert_allclose(W[b], w1, rtol=1e-12, atol=1e-14)
    parts = orc.chi2_parts(U, y, sig, w1, lam, nd)
    np.testing.assert_allclose(chi, parts[1], rtol=1e-12)
    assert cm == pytest.approx(parts[1], rel=1e-12)


def test_every_bootstrap_weight_set_is_optimal(orc):
    U, y, sig, nd = _problem(seed=8)
    lam = 0.5
    xi = inputs.bootstrap_noise(len(y), 20, 21)
    W, chi, cm = orc.bootstrap_solve(U, y, sig, lam, nd, xi)
    Ut = U / sig[:, None]
    H = Ut.T @ Ut + (2 * lam / U.shape[1]) * np.eye(U.shape[1])
    Yb = orc.bootstrap_data(y, sig, nd, xi)
    for b in range(20):
        q = Ut.T @ (Yb[b] / sig)
        k = orc.kkt_residual(H, q, W[b])
        assert k["neg_w"] == 0.0 and k["pg_inf"] <= 1e-9 * np.abs(q).max(), (b, k)
    # the weight sets differ (the data changed) and chi2_model lies between min and min + 2 ln B
    assert np.ptp(W, axis=0).max() > 1e-3
    assert chi.min() <= cm <= chi.min() + 2 * math.log(20)
