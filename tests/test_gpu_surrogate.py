"""GPU parity of the learned chi^2 emulator's kernels (forward, back-propagation,
Adam) against the FP64 oracle, and what delayed acceptance gains over plain
Metropolis on the exact model."""
import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

pytestmark = pytest.mark.gpu
SHAPE = (12, 64, 2)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2607_00117_gb300 import sw, surrogate
    sw.lib(build_if_missing=True)
    return torch, sw, surrogate


def _unflatten(p, shape):
    n_in, width, hidden = shape
    out, off = [], 0
    for l in range(hidden + 1):
        fin = n_in if l == 0 else width
        fout = 1 if l == hidden else width
        out.append(p[off:off + fout * fin].reshape(fout, fin).astype(np.float64)); off += fout * fin
        out.append(p[off:off + fout].astype(np.float64)); off += fout
    assert off == len(p)
    return out


def _setup(env, shape, B, seed):
    torch, sw, surrogate = env
    c = sw.Context(0, "fp32")
    emu = surrogate.Emulator(c, torch, shape, seed=seed)
    rng = np.random.default_rng(seed)
    # non-zero biases so that their gradients and the bias path are exercised
    p = emu.p.cpu().numpy()
    p += np.float32(0.05) * rng.standard_normal(len(p)).astype(np.float32)
    emu.p.copy_(torch.from_numpy(p))
    X = rng.uniform(-1, 1, (B, shape[0])).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    return c, emu, X, t


@pytest.mark.parametrize("shape,B", [(SHAPE, 1), (SHAPE, 37), (SHAPE, 300), ((12, 256, 3), 1), ((12, 256, 3), 300)])
def test_mlp_forward_and_gradient_vs_oracle(env, orc, shape, B):
    """Forward, BF16 inference and all gradients against the FP64 oracle, at a small network and at the
    configured emulator (12 -> 256 -> 256 -> 256 -> 1)."""
    torch, sw, surrogate = env
    SHAPE = shape
    c, emu, X, t = _setup(env, SHAPE, B, 7 + B)
    dev = emu.dev
    Xd, td = torch.from_numpy(X).to(dev), torch.from_numpy(t).to(dev)
    out = torch.empty(B, dtype=torch.float32, device=dev)
    c.mlp_forward(SHAPE, emu.p.data_ptr(), Xd.data_ptr(), B, out.data_ptr(), False)
    params = _unflatten(emu.p.cpu().numpy(), SHAPE)
    ref, _ = orc.mlp_forward(params, X.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-5)
    # BF16 inference: within BF16 rounding of the FP32 result
    c.mlp_forward(SHAPE, emu.p.data_ptr(), Xd.data_ptr(), B, out.data_ptr(), True)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=3e-2, atol=3e-2)
    loss = c.mlp_loss_grad(SHAPE, emu.p.data_ptr(), Xd.data_ptr(), td.data_ptr(), B, emu.g.data_ptr())
    loss_o, grads_o = orc.mlp_loss_grad(params, X.astype(np.float64), t.astype(np.float64))
    np.testing.assert_allclose(loss, loss_o, rtol=1e-5)
    g = _unflatten(emu.g.cpu().numpy(), SHAPE)
    for k, (a, b) in enumerate(zip(g, grads_o)):
        scale = np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() <= 1e-3 * scale, (k, np.abs(a - b).max(), scale)


def test_adam_vs_oracle(env, orc):
    torch, sw, surrogate = env
    c, emu, X, t = _setup(env, SHAPE, 64, 3)
    rng = np.random.default_rng(4)
    n = emu.n
    g = rng.standard_normal(n).astype(np.float32)
    p0 = emu.p.cpu().numpy().astype(np.float64)
    emu.g.copy_(torch.from_numpy(g))
    P, G, M, V = [p0.copy()], [g.astype(np.float64)], [np.zeros(n)], [np.zeros(n)]
    for step in (1, 2, 3):
        c.mlp_adam(n, emu.p.data_ptr(), emu.g.data_ptr(), emu.m.data_ptr(), emu.v.data_ptr(), step, 1e-3)
        orc.adam_step(P, G, M, V, step, lr=1e-3)
    np.testing.assert_allclose(emu.p.cpu().numpy(), P[0], rtol=0, atol=2e-6)


def test_training_fits_a_smooth_function(env):
    """Training by the library's kernels fits a smooth 12-D function: the
    held-out error falls well below the target's spread."""
    torch, sw, surrogate = env
    c = sw.Context(0, "fp32")
    emu = surrogate.Emulator(c, torch, (12, 128, 2), seed=11)
    rng = np.random.default_rng(12)
    u = rng.random((3000, 12))
    f = lambda uu: np.exp(1.0 + (uu[:, 0] - 0.4) ** 2 * 3 + np.sin(3 * uu[:, 1]) + 0.5 * uu[:, 2] * uu[:, 3])
    losses = emu.fit(u[:2500], f(u[:2500]), epochs=60, batch=128, lr=2e-3)
    assert losses[-1] < 0.05 * losses[0]
    pred = emu.predict(u[2500:], bf16=True)
    rel = np.abs(np.log(pred) - np.log(f(u[2500:])))
    assert np.median(rel) < 0.05, np.median(rel)


def test_delayed_acceptance_saves_exact_models(env, orc):
    """On the exact model (a small library over the 12-D box), delayed
    acceptance with the trained emulator runs far fewer exact models than plain
    Metropolis for the same number of steps, and a larger share of its exact
    models is accepted."""
    torch, sw, surrogate = env
    c = sw.Context(0, "fp32")
    grid = dict(inputs.WORKLOADS["barred_100k"]["grid"], nx=8, ny=8, pix=1.25, nR=5, nphi=6, nz=3, gh=1)
    truth = surrogate.box_point(np.full(12, 0.5))[0]
    mt = inputs.box_model(truth)
    ics = inputs.disc_ics(mt["potential"], 400, seed=901)
    S, dt = 200, 2 * inputs.DT_HALF_MYR
    # data: an independent library in the true model
    ics_d = inputs.disc_ics(mt["potential"], 400, seed=902)
    po = orc.make_pot(mt["potential"])
    gt = dict(grid, incl=mt["incl"], bar_angle=mt["bar_angle"])
    mom = orc.pixel_moments(po, mt["omega_p"], dt, S, ics_d, orc.make_obs(gt), np.ones(len(ics_d)))
    v0s, gh_err = inputs.gh_reference(mom)
    c.set_potential(mt["potential"])
    c.integrate_library(ics_d, mt["omega_p"], dt, S)
    Ud = c.project(gt, gh_v0s=v0s)
    Ug = Ud.copy().T.copy()
    Ud.free()
    y0 = Ug @ inputs.true_weights(len(ics_d), 903)
    sig = inputs.mock_sigma(y0, inputs.row_blocks(gt), gh_err=gh_err)
    y = y0 + sig * inputs.noise(len(y0), 904)
    exact = surrogate.ModelChi2(c, grid, ics, S, dt, y, sig, v0s)
    # training set from the exact model
    rng = np.random.default_rng(905)
    u_tr = np.clip(0.5 + 0.25 * rng.standard_normal((300, 12)), 0, 1)
    chi_tr = np.array([exact(surrogate.box_point(u)[0]) for u in u_tr])
    emu = surrogate.Emulator(c, torch, (12, 128, 2), seed=906)
    emu.fit(u_tr, chi_tr, epochs=150, batch=64, lr=2e-3)
    temp = np.sqrt(2 * len(y))
    n = 120
    exact.calls = 0
    mh = surrogate.mh_chain(exact, np.full(12, 0.5), n, 0.08, temp, seed=907)
    da = surrogate.da_chain(exact, emu, np.full(12, 0.5), n, 0.08, temp, seed=907)
    assert mh["n_exact"] == n + 1
    assert da["n_exact"] <= 0.7 * mh["n_exact"], (da, mh["n_exact"])
    assert da["n_accept"] / max(da["n_exact"] - 1, 1) > mh["n_accept"] / n
