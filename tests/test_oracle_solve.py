"""Pins for the oracle's weight problem (Sec. 2.3 Eq. objective_function and its
compact NNLS form; Sec. 2.4 chi^2) and for the emulator MLP.

* brute-force enumeration of every support on tiny problems (the strictly
  convex problem has one minimiser) against Lawson-Hanson in both forms, the
  paper's ADMM, and SciPy's NNLS on the stacked system;
* noise-free data with a full-rank U and positive weights gives chi^2 = 0;
* the KKT certificate and the strong-convexity bound on medium problems;
* the MLP's hand-written gradient against central finite differences.
"""
import numpy as np
import pytest
import scipy.optimize


def _problem(seed, M, N, lam, density=0.5):
    rng = np.random.default_rng(seed)
    U = rng.random((M, N)) * (rng.random((M, N)) < density)
    w_true = 2 * rng.random(N)
    y0 = U @ w_true
    sigma = 0.02 * np.maximum(y0, 0.01 * y0.mean()) + 1e-3
    y = y0 + sigma * rng.standard_normal(M) * 5
    return U, y, sigma


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_bruteforce_vs_lawson_hanson(orc, seed, lam):
    M, N = 24, 10
    U, y, sigma = _problem(seed, M, N, lam)
    Ut, yt = orc.whiten(U, y, sigma)
    H, q = orc.normal_equations(Ut, yt, lam)
    w_bf = orc.nnls_bruteforce(H, q)
    A = np.vstack([Ut, np.sqrt(2 * lam / N) * np.eye(N)])
    b = np.concatenate([yt, np.zeros(N)])
    w_lh = orc.nnls_lawson_hanson(A, b)
    w_ne = orc.nnls_lh_normal(H, q)
    w_sp = scipy.optimize.nnls(A, b)[0]
    w_ad, _ = orc.admm_nnls(H, q, tol=1e-13)
    s = max(1.0, np.abs(w_bf).max())
    for w in (w_lh, w_ne, w_sp, w_ad):
        np.testing.assert_allclose(w, w_bf, atol=1e-8 * s)
    f = orc.objective(H, q, w_bf)
    assert orc.objective(H, q, w_lh) == pytest.approx(f, rel=1e-12, abs=1e-12)


def test_noise_free_full_rank_gives_zero_chi2(orc):
    rng = np.random.default_rng(5)
    M, N = 60, 20
    U = rng.random((M, N))
    w_true = 0.5 + rng.random(N)
    y = U @ w_true
    sigma = 0.02 * y
    Ut, yt = orc.whiten(U, y, sigma)
    H, q = orc.normal_equations(Ut, yt, 0.0)
    w = orc.nnls_lh_normal(H, q)
    np.testing.assert_allclose(w, w_true, rtol=1e-8)
    chi2 = orc.chi2_parts(U, y, sigma, w, 0.0, 0)
    assert chi2[0] < 1e-12


def test_kkt_certificate_medium(orc):
    M, N, lam = 400, 150, 1.0
    U, y, sigma = _problem(9, M, N, lam, density=0.2)
    Ut, yt = orc.whiten(U, y, sigma)
    H, q = orc.normal_equations(Ut, yt, lam)
    w = orc.nnls_lh_normal(H, q)
    k = orc.kkt_residual(H, q, w)
    scale = np.abs(q).max()
    assert k["neg_w"] == 0.0 and k["pg_inf"] <= 1e-10 * scale and k["compl"] <= 1e-9 * scale * max(1, w.max())
    # strong convexity: f(w) - f* <= ||P(g)||^2 / (2 mu), mu = 2 lam / N; check against
    # the same solution perturbed (f increases by at most the bound)
    w2 = np.maximum(0, w + 1e-3 * np.random.default_rng(1).standard_normal(N))
    k2 = orc.kkt_residual(H, q, w2)
    gap = orc.objective(H, q, w2) - orc.objective(H, q, w)
    assert 0 <= gap <= k2["pg_norm2"] / (2 * 2 * lam / N) * (1 + 1e-9)
    w_ad, it = orc.admm_nnls(H, q, tol=1e-12)
    f = orc.objective(H, q, w)
    assert orc.objective(H, q, w_ad) == pytest.approx(f, rel=1e-9)


def test_chi2_parts_definition(orc):
    rng = np.random.default_rng(2)
    U = rng.random((10, 4)); y = rng.random(10); s = 0.1 + rng.random(10); w = rng.random(4)
    c = orc.chi2_parts(U, y, s, w, 2.0, n_dens=3)
    r = [(sum(U[i, j] * w[j] for j in range(4)) - y[i]) / s[i] for i in range(10)]
    assert c[0] == pytest.approx(sum(v * v for v in r))
    assert c[1] == pytest.approx(sum(v * v for v in r[3:]))
    assert c[2] == pytest.approx(2.0 / 4 * sum(v * v for v in w))


def _mlp_params(rng, sizes=(12, 256, 256, 256, 1)):
    p = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        p.append(rng.standard_normal((b, a)) / np.sqrt(a))
        p.append(0.1 * rng.standard_normal(b))
    return p


def test_mlp_gradient_vs_finite_differences(orc):
    rng = np.random.default_rng(4)
    params = _mlp_params(rng, (12, 16, 16, 16, 1))
    X = rng.standard_normal((7, 12)); t = rng.standard_normal(7)
    loss, grads = orc.mlp_loss_grad(params, X, t)
    h = 1e-6
    for k in range(len(params)):
        flat = params[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h; lp, _ = orc.mlp_loss_grad(params, X, t)
            flat[i] = old - h; lm, _ = orc.mlp_loss_grad(params, X, t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert grads[k].reshape(-1)[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_mlp_shapes_and_adam(orc):
    rng = np.random.default_rng(8)
    params = _mlp_params(rng)
    assert sum(p.size for p in params) == 12 * 256 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    X = rng.standard_normal((32, 12)); t = rng.standard_normal(32)
    m = [np.zeros_like(p) for p in params]; v = [np.zeros_like(p) for p in params]
    loss0, g = orc.mlp_loss_grad(params, X, t)
    p0 = [q.copy() for q in params]
    orc.adam_step(params, g, m, v, 1, lr=1e-3)
    # first Adam step moves every coordinate by lr * sign(g) (bias-corrected m/sqrt(v) = g/|g|)
    for a, b, gg in zip(params, p0, g):
        nz = np.abs(gg) > 1e-4   # eps = 1e-8 matters below that
        np.testing.assert_allclose((b - a)[nz], 1e-3 * np.sign(gg[nz]), rtol=1e-3)
    for it in range(2, 60):
        _, g = orc.mlp_loss_grad(params, X, t)
        orc.adam_step(params, g, m, v, it, lr=1e-3)
    loss1, _ = orc.mlp_loss_grad(params, X, t)
    assert loss1 < 0.5 * loss0


@pytest.mark.parametrize("seed", range(4))
def test_whiten_pins_the_objective(orc, seed):
    """whiten (with normal_equations) against the objective's definition: at any w,
    1/2 w^T H w - q^T w + 1/2 |y~|^2 equals 1/2 ||(U w - y)/sigma||^2 + (lam/N) |w|^2,
    with chi^2 and the regulariser taken from chi2_parts.  Errors far from 1 make a
    division by sigma^2 (or by sqrt(sigma)) fail; a hand case fixes the scaling."""
    rng = np.random.default_rng(40 + seed)
    M, N, lam = 30, 12, 0.7
    U = rng.random((M, N))
    y = rng.random(M) * 3.0
    sigma = rng.uniform(0.05, 9.0, M)
    Ut, yt = orc.whiten(U, y, sigma)
    H, q = orc.normal_equations(Ut, yt, lam)
    for _ in range(3):
        w = rng.uniform(0, 2, N)
        f = orc.objective(H, q, w) + 0.5 * yt @ yt
        c = orc.chi2_parts(U, y, sigma, w, lam, 5)
        assert abs(f - (0.5 * c[0] + c[2])) <= 1e-12 * max(1.0, f)
    Ut2, yt2 = orc.whiten(np.array([[2.0, 4.0], [3.0, 9.0]]), np.array([6.0, 12.0]), np.array([2.0, 3.0]))
    np.testing.assert_array_equal(Ut2, [[1.0, 2.0], [1.0, 3.0]])
    np.testing.assert_array_equal(yt2, [3.0, 4.0])
