"""Pins for the oracle's Dehnen-Aly barred components (Sec. 2.1.2, App. A, Eq.
Rn_to_In): the parent T3 and V4 pairs with R^-n replaced by the needle integral I_n.

Closed forms: I_1 for the flat needle (eta = 0) and for the triangular one
(eta = 1); the T3 family with a = 0 is the Miyamoto-Nagai disc, and its flat-needle
bar must equal the Long-Murali closed form of oracle.c; a vanishing needle returns
the parent pair.  Invariants: Poisson's equation for the barred T3 long bar and V4
bulge at the paper's parameters, and the bar's reflection symmetries.
"""
import math

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

G = 4.300917e-6


def _pts(seed=4, n=6):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-6, 6, n), rng.uniform(-4, 4, n), rng.uniform(-2, 2, n)], 1)


def test_needle_integral_closed_forms(orc):
    L = 3.0
    p = _pts()
    x, y, Z = p[:, 0], p[:, 1], 0.7 + np.abs(p[:, 2])
    q = np.sqrt(y * y + Z * Z)
    flat = (np.arcsinh((x + L) / q) - np.arcsinh((x - L) / q)) / (2 * L)
    np.testing.assert_allclose(orc.needle_In(x, y, Z, 1, L, 0.0), flat, rtol=1e-12)
    # triangular needle f(u) = (1 - |u|/L)/L: with A = asinh(x'/q), S = sqrt(x'^2 + q^2),
    # int (1 - (x - x')/L) dx'/S over [x - L, x] and int (1 - (x' - x)/L) dx'/S over [x, x + L]
    A = lambda t: np.arcsinh(t / q)
    S = lambda t: np.sqrt(t * t + q * q)
    left = (A(x) - A(x - L)) - ((x * (A(x) - A(x - L))) - (S(x) - S(x - L))) / L
    right = (A(x + L) - A(x)) - ((S(x + L) - S(x)) - x * (A(x + L) - A(x))) / L
    np.testing.assert_allclose(orc.needle_In(x, y, Z, 1, L, 1.0), (left + right) / L, rtol=1e-12)


def test_flat_needle_t3_with_a_zero_is_long_murali(orc):
    M, c, L = 1e10, 0.5, 4.0
    pts = _pts(seed=9, n=8)
    phi_da, _ = orc.dehnen_aly("T3", M, 0.0, c, L, 0.0, pts)
    pot = orc.make_pot(dict(disc_M=0.0, bar_M=M, bar_L=L, bar_b=0.0, bar_c=c))
    phi_lm, _ = orc.potential(pot, pts, orc.BAR)
    np.testing.assert_allclose(phi_da, phi_lm, rtol=1e-11)


@pytest.mark.parametrize("family", ["T3", "V4"])
def test_vanishing_needle_gives_the_parent(orc, family):
    pts = _pts(seed=2)
    p0, r0 = orc.dehnen_aly(family, 1e10, 0.8, 0.5, 0.0, 0.0, pts)
    for eta in (0.0, 1.0):
        p1, r1 = orc.dehnen_aly(family, 1e10, 0.8, 0.5, 1e-5, eta, pts)
        np.testing.assert_allclose(p1, p0, rtol=1e-8)
        np.testing.assert_allclose(r1, r0, rtol=1e-8)


def _laplacian(f, p, h=4e-3):
    """Central second differences with one Richardson step (the h^2 error removed)."""
    def lap(hh):
        out = np.zeros(len(p))
        f0 = f(p)
        for k in range(3):
            e = np.zeros(3); e[k] = hh
            out += (f(p + e) - 2 * f0 + f(p - e)) / (hh * hh)
        return out
    return (4 * lap(0.5 * h) - lap(h)) / 3


@pytest.mark.parametrize("family,a,b,L,eta", [("T3", 0.8, 0.3, 4.0, 1.0), ("V4", 0.5, 0.5, 0.1, 0.0),
                                              ("T3", 1.0, 0.5, 3.0, -0.5)])
def test_poisson_for_barred_components(orc, family, a, b, L, eta):
    M = 1e10
    pts = _pts(seed=13, n=8)
    lap = _laplacian(lambda q: orc.dehnen_aly(family, M, a, b, L, eta, q)[0], pts)
    _, rho = orc.dehnen_aly(family, M, a, b, L, eta, pts)
    np.testing.assert_allclose(lap, 4 * math.pi * G * rho, rtol=1e-4)   # the differences' rounding floor


def test_bar_symmetries_and_paper_composite(orc):
    p = _pts(seed=21)
    phi, rho = orc.paper_bar(1e10, 4.0, 0.3, p)
    for s in ([-1, 1, 1], [1, -1, 1], [1, 1, -1]):
        ph2, rh2 = orc.paper_bar(1e10, 4.0, 0.3, p * np.array(s))
        np.testing.assert_allclose(ph2, phi, rtol=1e-13)
        np.testing.assert_allclose(rh2, rho, rtol=1e-13)
    # far away the composite is a point mass M_b
    far = np.array([[300.0, 40.0, 20.0]])
    ph, _ = orc.paper_bar(1e10, 4.0, 0.3, far)
    assert ph[0] == pytest.approx(-G * 1e10 / np.linalg.norm(far), rel=1e-3)
    # the bar is elongated along x: deeper potential at (2, 0, 0) than at (0, 2, 0)
    a, _ = orc.paper_bar(1e10, 4.0, 0.3, np.array([[2.0, 0, 0], [0, 2.0, 0]]))
    assert a[0] < a[1]


@pytest.mark.parametrize("n", [1, 3, 5, 7, 9, 11, 13])
def test_closed_form_needle_integrals_match_quadrature(orc, n):
    """The antiderivative recurrences against the quadrature; for the 0.1 kpc needle of
    the V4 bulge the closed form loses digits to cancellation (differences of nearly equal
    antiderivatives), which the looser bound records."""
    rng = np.random.default_rng(1)
    x, y, Z = rng.uniform(-6, 6, 30), rng.uniform(-4, 4, 30), 0.6 + rng.uniform(0, 2, 30)
    for eta in (-0.5, 0.0, 1.0):
        np.testing.assert_allclose(orc.needle_In_closed(x, y, Z, n, 4.0, eta), orc.needle_In(x, y, Z, n, 4.0, eta),
                                   rtol=1e-10)
        np.testing.assert_allclose(orc.needle_In_closed(x, y, Z, n, 0.1, eta), orc.needle_In(x, y, Z, n, 0.1, eta),
                                   rtol=1e-5)


PAPER_BAR_POT = dict(inputs.DISC_HALO, bar_M=1e10, bar_L=4.0, bar_kind=1)


def test_c_oracle_paper_bar_matches_and_is_consistent(orc):
    """oracle.c's paper bar (bar_kind = 1, used by its integrator) against the Python
    implementation, its acceleration against -grad Phi, and Poisson's equation."""
    pot = orc.make_pot(PAPER_BAR_POT)
    pts = _pts(seed=31, n=10)
    phi_c, acc_c = orc.potential(pot, pts, orc.BAR)
    rho_c = orc.density(pot, pts, orc.BAR)
    phi_p, rho_p = orc.paper_bar(1e10, 4.0, inputs.DISC_HALO["disc_b"], pts)
    np.testing.assert_allclose(phi_c, phi_p, rtol=1e-12)
    np.testing.assert_allclose(rho_c, rho_p, rtol=1e-12)
    h = 1e-4
    for k in range(3):
        e = np.zeros(3); e[k] = h
        fd = -(orc.potential(pot, pts + e, orc.BAR)[0] - orc.potential(pot, pts - e, orc.BAR)[0]) / (2 * h)
        np.testing.assert_allclose(acc_c[:, k], fd, rtol=1e-6, atol=1e-7 * np.abs(acc_c).max())
    lap = _laplacian(lambda q: orc.potential(pot, q, orc.BAR)[0], pts)
    np.testing.assert_allclose(lap, 4 * math.pi * G * rho_c, rtol=1e-4)


def test_jacobi_energy_in_the_rotating_paper_bar(orc):
    """Disc + halo + the paper's bar rotating at 40 km/s/kpc: the fixed-step KDK keeps the
    Jacobi energy bounded with no secular drift, as for the Long-Murali bar."""
    pot = orc.make_pot(PAPER_BAR_POT)
    omega, dt, S = 40.0, inputs.DT_HALF_MYR, 20_000
    ic = inputs.disc_ics(inputs.DISC_HALO, 1, seed=21, vfrac=(1.0, 1.0), sigma_v=5.0)[0]
    tr = orc.trajectory(pot, omega, dt, S, ic)
    ej = np.array([orc.jacobi(pot, omega, n * dt, tr[n]) for n in range(0, S + 1, 20)])
    dev = np.abs(ej / ej[0] - 1)
    assert dev.max() < 1e-4, dev.max()
    half = len(dev) // 2
    assert dev[half:].max() < 3 * max(dev[:half].max(), 1e-12)
