"""The preconditioner of the weight solve's reduced systems on its own: the Cholesky factor L
and the explicit inverse X = L^{-1} of a shifted, Jacobi-scaled passive Gram (the matrices the
active set factors; Sec. 2.3, solved here by preconditioned conjugate gradients), through
sw_factor_preconditioner.

Sizes: one diagonal block (K = 77, 128: only the 128-wide diagonal kernel runs), a ragged
blocked case (K = 300: 128 + 128 + 44) and a larger one (K = 1 000).  The gates are backward
errors, which hold whatever the matrix's condition (these reach 1e4-1e5, like the passive
systems): ||G - L L^T||_F <= tol ||G||_F and ||X L - I||_F <= tol || |X| |L| ||_F, with tol =
(K + 2) u_32 for FP32 arithmetic (mode 1, and mode 0 on a single block) and 2^-16 sqrt(K) +
(K + 2) u_32 for the tensor-core updates (each BF16 hi + lo product is exact to 2^-16 of
|a||b|, and the sum of |L_ik L_jk| over k is at most sqrt(G_ii G_jj) = 1).  A misplaced index
gives residuals of order one.  The FP64 factor of the same FP32 matrix is printed beside them."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    return swmod.Context(0, "fp32")


def passive_gram(K, seed, M=None):
    """S (A^T A) S + ridge with near-duplicate column pairs (bundled orbits of one family), S the
    Jacobi scaling, as the active set forms it; returned in FP32."""
    rng = np.random.default_rng(seed)
    M = M or 2 * K + 50
    A = np.abs(rng.standard_normal((M, K))) * rng.uniform(0.2, 3.0, K)
    A[:, 1::2] = A[:, 0:K - K % 2:2][:, :A[:, 1::2].shape[1]] + 0.3 * np.abs(rng.standard_normal((M, K // 2)))
    H = A.T @ A
    s = 1.0 / np.sqrt(np.diag(H))
    G = (s[:, None] * H * s[None, :]) + 1e-3 * np.eye(K)
    return G.astype(np.float32)


U32 = 2.0 ** -24


def _errs(G32, L, X):
    Gd = np.tril(G32.astype(np.float64))
    Gd = Gd + np.tril(Gd, -1).T
    Lg = np.tril(L.astype(np.float64))
    Xg = X.astype(np.float64)
    back_L = np.linalg.norm(Gd - Lg @ Lg.T) / np.linalg.norm(Gd)
    back_X = np.linalg.norm(Xg @ Lg - np.eye(len(Gd))) / np.linalg.norm(np.abs(Xg) @ np.abs(Lg))
    Le = np.linalg.cholesky(Gd)
    fwd_L = np.linalg.norm(Lg - Le) / np.linalg.norm(Le)
    return back_L, back_X, fwd_L, np.linalg.cond(Gd), np.abs(np.triu(Xg, 1)).max()


@pytest.mark.parametrize("K,mode", [(77, 0), (128, 0), (300, 0), (1000, 0), (300, 1), (1000, 1)])
def test_factor_backward_error(ctx, K, mode):
    G = passive_gram(K, 7000 + K)
    L, X, info = ctx.factor_preconditioner(G, mode)
    assert info == 0
    back_L, back_X, fwd_L, cond, upper = _errs(G, L, X)
    tol = (K + 2) * U32 + (2.0 ** -16 * np.sqrt(K) if mode == 0 and K > 128 else 0.0)
    print(f"K={K} mode={mode}: cond {cond:.3g}; backward |G-LL^T|/|G| {back_L:.3g}, |XL-I|/||X||L|| {back_X:.3g} "
          f"(tol {tol:.3g}); forward |L-L*|/|L*| {fwd_L:.3g}")
    assert upper == 0.0
    assert back_L <= tol and back_X <= tol


def test_factor_input_upper_triangle_ignored(ctx):
    """Only the lower triangle is read: garbage above the diagonal changes nothing."""
    G = passive_gram(300, 7100)
    Gg = G.copy()
    Gg[np.triu_indices(300, 1)] = np.float32(np.nan)
    L0, X0, _ = ctx.factor_preconditioner(G, 0)
    L1, X1, _ = ctx.factor_preconditioner(Gg, 0)
    np.testing.assert_array_equal(np.tril(L0), np.tril(L1))
    np.testing.assert_array_equal(X0, X1)


def test_factor_reports_nonpositive_pivot(ctx):
    G = passive_gram(200, 7200).astype(np.float64)
    G[150, :150] = 0.0
    G[150, 150] = -1.0                     # pivot 151 negative
    L, X, info = ctx.factor_preconditioner(G.astype(np.float32), 0)
    assert info == 151
    L, X, info = ctx.factor_preconditioner(G.astype(np.float32), 1)
    assert info == 151


@pytest.mark.parametrize("K", [300, 640, 1000])
@pytest.mark.parametrize("variant", [(0, 0), (1, 0), (1, 1)])
def test_factor_step_variants(K, variant):
    """The tensor-core form's schedules: 128-wide steps (chol_super 0), 256-wide super-steps with
    rank-256 bulk updates and SIMT panels (1, chol_panel_tc 0) or panels on the tensor cores (1, 1).
    Each meets the tensor-core gate; the variants agree with one another to it."""
    from paper_2607_00117_gb300 import sw as swmod
    swmod.lib(build_if_missing=True)
    G = passive_gram(K, 7200 + K)
    c = swmod.Context(0, "fp32")
    c.set_option("chol_super", variant[0])
    c.set_option("chol_panel_tc", variant[1])
    L, X, info = c.factor_preconditioner(G, 0)
    assert info == 0
    back_L, back_X, fwd_L, cond, upper = _errs(G, L, X)
    tol = (K + 2) * U32 + 2.0 ** -16 * np.sqrt(K)
    print(f"K={K} super={variant[0]} panel_tc={variant[1]}: backward {back_L:.3g}, {back_X:.3g} (tol {tol:.3g}); "
          f"forward {fwd_L:.3g}")
    assert upper == 0.0
    assert back_L <= tol and back_X <= tol
