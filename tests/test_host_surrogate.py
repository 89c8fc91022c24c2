"""Host logic of the delayed-acceptance sampler, on the CPU (no GPU, no network).

Delayed acceptance (Christen & Fox 2005) screens each proposal with the
emulated chi^2 and lets the exact chi^2 decide, with a second-stage ratio that
divides out the screen; the chain then targets the exact posterior whatever
the emulator.  Here the exact chi^2 is a known function of the unit-box point
(an isotropic Gaussian of width 0.12 about the box centre, so the posterior
exp(-chi^2 / 2) is that Gaussian truncated at 4.2 sigma, standard deviation
0.1199 per coordinate) and the emulators are deliberately wrong in scale and
shape.  Without the second-stage correction the chain would sample
exp(-(1 + s) chi^2 / 2) for an emulator s chi^2 and come out 18 % too narrow
with s = 0.5, far outside the tolerances below.
"""
import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs, surrogate

MU, SD = 0.5, 0.12
SD_TRUNC = 0.1199          # standard deviation of N(0.5, 0.12^2) truncated to [0, 1]
STEPS, BURN, STEP, SEED = 20000, 2000, 0.06, 1


def exact_chi2(theta):
    u = inputs.box_unit(theta)[0]
    return float(np.sum(((u - MU) / SD) ** 2))


class Emulator:
    """Stand-in for the network: s * chi^2 + a * sin(7 u_0)."""

    def __init__(self, scale, wiggle):
        self.scale, self.wiggle = scale, wiggle

    def predict(self, u):
        u = np.atleast_2d(u)
        return self.scale * np.sum(((u - MU) / SD) ** 2, axis=1) + self.wiggle * np.sin(7.0 * u[:, 0])


def _moments(chain):
    c = chain[BURN:]
    return np.abs(c.mean(0) - MU), c.std(0)


def test_box_point_inverts_box_unit():
    u = np.random.default_rng(3).random((5, 12))
    np.testing.assert_allclose(inputs.box_unit(surrogate.box_point(u)), u, rtol=0, atol=1e-12)


def test_reflection_keeps_points_in_the_box():
    x = np.array([-0.3, 0.2, 1.4, 2.6, -1.7])
    np.testing.assert_allclose(surrogate._reflect(x), [0.3, 0.2, 0.6, 0.6, 0.3], atol=1e-12)


@pytest.mark.parametrize("scale,wiggle", [(1.0, 0.5), (0.5, 3.0)])
def test_delayed_acceptance_targets_the_exact_posterior(scale, wiggle):
    u0 = np.full(12, 0.5)
    r = surrogate.da_chain(exact_chi2, Emulator(scale, wiggle), u0, STEPS, STEP, 1.0, SEED)
    dev, sd = _moments(r["chain"])
    assert dev.mean() < 0.012 and dev.max() < 0.03, dev
    assert abs(sd.mean() - SD_TRUNC) < 0.006 and np.all(np.abs(sd - SD_TRUNC) < 0.015), sd
    # every proposal the screen passes costs one exact model, and only those
    assert r["n_exact"] == r["n_stage1"] + 1


def test_plain_metropolis_targets_the_same_posterior():
    r = surrogate.mh_chain(exact_chi2, np.full(12, 0.5), STEPS, STEP, 1.0, SEED)
    dev, sd = _moments(r["chain"])
    assert dev.mean() < 0.012 and abs(sd.mean() - SD_TRUNC) < 0.006
    assert r["n_exact"] == STEPS + 1


def test_informative_screen_saves_exact_models():
    """With an emulator close to the exact chi^2 the screen rejects most of the
    proposals the exact model would reject: far fewer exact models for about
    the same number of accepted moves."""
    u0 = np.full(12, 0.5)
    da = surrogate.da_chain(exact_chi2, Emulator(1.0, 0.5), u0, STEPS, STEP, 1.0, SEED)
    mh = surrogate.mh_chain(exact_chi2, u0, STEPS, STEP, 1.0, SEED)
    assert da["n_exact"] < 0.5 * mh["n_exact"]
    assert da["n_accept"] > 0.85 * mh["n_accept"]
