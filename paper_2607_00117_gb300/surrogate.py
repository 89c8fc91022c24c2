"""Learned chi^2 emulator and delayed-acceptance MCMC over the 12-D potential box.

The paper samples its 12 potential parameters by MCMC on the exact chi^2 of
each model (Sec. 3.2: 1.3 s per evaluation, 32 chains x 1 500 steps) and points
to surrogates as the way to cheaper likelihoods (Sec. 5.3).  Here a fully
connected network (12 -> 256 -> 256 -> 256 -> 1, SiLU) learns the standardised
log chi^2 over the box from models the pipeline itself computes; its training
and inference run in the library's own kernels (`sw_mlp_*`).  It screens
proposals in a delayed-acceptance Metropolis sampler (Christen & Fox 2005): a
proposal that the emulator rejects costs no exact model, and every proposal the
emulator passes is judged by the exact chi^2, so the chain targets the exact
posterior.

This module is host logic only (argument marshalling, the Markov chain); the
network's arithmetic and every model evaluation run in CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs
from . import sw

SHAPE = (12, 256, 3)          # n_in, width, hidden layers


class Emulator:
    """The network and its Adam state on one context's device (torch tensors
    provide the device memory)."""

    def __init__(self, ctx: "sw.Context", torch, shape=SHAPE, seed: int = 0):
        self.ctx, self.torch, self.shape = ctx, torch, tuple(shape)
        n = int(sw.lib().sw_mlp_param_count(*self.shape))
        if n <= 0:
            raise ValueError(f"invalid network shape {shape}")
        self.n = n
        rng = np.random.Generator(np.random.PCG64(seed))
        p = np.zeros(n, dtype=np.float32)
        off = 0
        n_in, width, hidden = self.shape
        for l in range(hidden + 1):
            fin = n_in if l == 0 else width
            fout = 1 if l == hidden else width
            bound = 1.0 / math.sqrt(fin)
            p[off:off + fout * fin] = rng.uniform(-bound, bound, fout * fin)
            off += fout * fin + fout                    # biases start at zero
        dev = torch.device("cuda", ctx.device)
        self.dev = dev
        self.p = torch.from_numpy(p).to(dev)
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.step = 0
        self.t_mu, self.t_sd = 0.0, 1.0

    @staticmethod
    def features(u: np.ndarray) -> np.ndarray:
        """Unit-box coordinates -> network inputs in [-1, 1]."""
        return np.ascontiguousarray(2.0 * np.atleast_2d(u) - 1.0, dtype=np.float32)

    def fit(self, u: np.ndarray, chi2: np.ndarray, epochs: int = 200, batch: int = 256, lr: float = 1e-3,
            seed: int = 1) -> list:
        """Train on (unit-box point, chi^2) pairs; the target is the standardised
        log chi^2.  Returns the mean loss of each epoch."""
        torch = self.torch
        t = np.log(np.asarray(chi2, dtype=np.float64))
        self.t_mu, self.t_sd = float(t.mean()), float(t.std() or 1.0)
        X = torch.from_numpy(self.features(u)).to(self.dev)
        T = torch.from_numpy(((t - self.t_mu) / self.t_sd).astype(np.float32)).to(self.dev)
        rng = np.random.Generator(np.random.PCG64(seed))
        n = len(t)
        losses = []
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).to(self.dev)
            tot, cnt = 0.0, 0
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                xb, tb = X[idx].contiguous(), T[idx].contiguous()
                loss = self.ctx.mlp_loss_grad(self.shape, self.p.data_ptr(), xb.data_ptr(), tb.data_ptr(), len(idx),
                                              self.g.data_ptr())
                self.step += 1
                self.ctx.mlp_adam(self.n, self.p.data_ptr(), self.g.data_ptr(), self.m.data_ptr(),
                                  self.v.data_ptr(), self.step, lr)
                tot += loss * len(idx)
                cnt += len(idx)
            losses.append(tot / cnt)
        return losses

    def predict(self, u: np.ndarray, bf16: bool = True) -> np.ndarray:
        """Emulated chi^2 at unit-box points (BF16 inference by default)."""
        torch = self.torch
        X = torch.from_numpy(self.features(u)).to(self.dev)
        out = torch.empty(len(X), dtype=torch.float32, device=self.dev)
        self.ctx.mlp_forward(self.shape, self.p.data_ptr(), X.data_ptr(), len(X), out.data_ptr(), bf16)
        z = out.cpu().numpy().astype(np.float64)
        return np.exp(z * self.t_sd + self.t_mu)


class ModelChi2:
    """Exact chi^2_obs of one trial point of the 12-D box: the potential, pattern
    speed and viewing angles come from the point, the orbit library is
    integrated, projected to GH rows and solved against fixed data."""

    def __init__(self, ctx: "sw.Context", grid: dict, ics: np.ndarray, nsteps: int, dt: float, y: np.ndarray,
                 sigma: np.ndarray, gh_v0s: np.ndarray, lam: float = 1.0):
        self.ctx, self.grid, self.ics, self.S, self.dt = ctx, dict(grid), ics, nsteps, dt
        self.y, self.sigma, self.v0s, self.lam = y, sigma, gh_v0s, lam
        self.calls = 0

    def __call__(self, theta: np.ndarray) -> float:
        m = inputs.box_model(theta)
        c = self.ctx
        c.set_potential(m["potential"])
        c.integrate_library(self.ics, m["omega_p"], self.dt, self.S)
        g = dict(self.grid, incl=m["incl"], bar_angle=m["bar_angle"])
        U = c.project(g, gh_v0s=self.v0s)
        _, chi2 = c.solve_weights(U, self.y, self.sigma, self.lam, allow_nonconv=True)
        U.free()
        self.calls += 1
        return float(chi2[1])


def box_point(u: np.ndarray) -> np.ndarray:
    """Unit-box coordinates -> box parameters (inverse of inputs.box_unit)."""
    u = np.atleast_2d(u)
    out = np.empty_like(u, dtype=np.float64)
    for j, k in enumerate(inputs.BOX_KEYS):
        lo, hi, kind = inputs.BOX[k]
        out[:, j] = np.exp(np.log(lo) + u[:, j] * (np.log(hi) - np.log(lo))) if kind == "log" else lo + u[:, j] * (hi - lo)
    return out


def _reflect(u: np.ndarray) -> np.ndarray:
    """Fold a random-walk step back into [0, 1] (keeps the proposal symmetric)."""
    u = np.mod(u, 2.0)
    return np.where(u > 1.0, 2.0 - u, u)


def mh_chain(exact, u0: np.ndarray, n_steps: int, step: float, temp: float, seed: int) -> dict:
    """Plain random-walk Metropolis on exp(-chi^2 / (2 temp)) with a uniform
    prior on the unit box: one exact model per step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = np.array(u0, dtype=np.float64)
    c = exact(box_point(u)[0])
    n_exact, n_acc = 1, 0
    chain = [u.copy()]
    for _ in range(n_steps):
        up = _reflect(u + step * rng.standard_normal(u.shape))
        cp = exact(box_point(up)[0])
        n_exact += 1
        if math.log(rng.random() + 1e-300) < -(cp - c) / (2 * temp):
            u, c = up, cp
            n_acc += 1
        chain.append(u.copy())
    return {"chain": np.array(chain), "n_exact": n_exact, "n_accept": n_acc}


def da_chain(exact, emu: Emulator, u0: np.ndarray, n_steps: int, step: float, temp: float, seed: int) -> dict:
    """Delayed-acceptance Metropolis (Christen & Fox 2005): stage 1 accepts the
    proposal with min(1, exp(-(e' - e) / 2T)) on the emulated chi^2 e; stage 2
    runs the exact model and accepts with
    min(1, exp(-(c' - c) / 2T) * exp((e' - e) / 2T)), which makes the chain
    reversible for the exact posterior."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = np.array(u0, dtype=np.float64)
    c = exact(box_point(u)[0])
    e = float(emu.predict(u[None, :])[0])
    n_exact, n_acc, n_stage1 = 1, 0, 0
    chain = [u.copy()]
    for _ in range(n_steps):
        up = _reflect(u + step * rng.standard_normal(u.shape))
        ep = float(emu.predict(up[None, :])[0])
        if math.log(rng.random() + 1e-300) >= -(ep - e) / (2 * temp):
            chain.append(u.copy())
            continue
        n_stage1 += 1
        cp = exact(box_point(up)[0])
        n_exact += 1
        if math.log(rng.random() + 1e-300) < -(cp - c) / (2 * temp) + (ep - e) / (2 * temp):
            u, c, e = up, cp, ep
            n_acc += 1
        chain.append(u.copy())
    return {"chain": np.array(chain), "n_exact": n_exact, "n_accept": n_acc, "n_stage1": n_stage1}
