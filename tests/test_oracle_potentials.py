"""Pins for the oracle's potentials and forces (Sec. 3.2.1-3.2.2, Eq. Rn_to_In).

Each check compares the oracle with something other than itself: the paper's
printed densities through Poisson's equation, numerical differentiation,
numerical quadrature of the needle convolution, and NFW's defining identities.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from paper_2607_00117_gb300 import inputs

G = 4.300917e-6


def _pot(orc, **kw):
    p = dict(inputs.DISC_HALO, **inputs.BAR)
    p.update(kw)
    return orc.make_pot(p)


def _laplacian(orc, pot, x, mask, h):
    lap = np.zeros(len(x))
    phi0, _ = orc.potential(pot, x, mask)
    for k in range(3):
        e = np.zeros(3); e[k] = h
        pp, _ = orc.potential(pot, x + e, mask)
        pm, _ = orc.potential(pot, x - e, mask)
        lap += (pp - 2 * phi0 + pm) / (h * h)
    return lap


def _points(n, seed, Rmax=8.0, zmax=1.5):
    rng = np.random.default_rng(seed)
    R = Rmax * np.sqrt(rng.random(n)) + 0.2
    ph = 2 * np.pi * rng.random(n)
    z = zmax * (2 * rng.random(n) - 1)
    return np.stack([R * np.cos(ph), R * np.sin(ph), z], 1)


@pytest.mark.parametrize("mask_name", ["DISC", "HALO", "BAR"])
def test_poisson(orc, mask_name):
    """lap Phi = 4 pi G rho for each component against the paper's printed rho
    (MN, NFW) and, for the bar, against the needle convolution of MN's rho."""
    pot = _pot(orc)
    mask = getattr(orc, mask_name)
    x = _points(200, 11)
    lap = 0.5 * (_laplacian(orc, pot, x, mask, 2e-3) * 4 - _laplacian(orc, pot, x, mask, 4e-3)) / 1.5  # Richardson
    rho = orc.density(pot, x, mask, bar_nodes=256)
    np.testing.assert_allclose(lap, 4 * np.pi * G * rho, rtol=2e-6)


def test_poisson_plummer(orc):
    pot = orc.make_pot(dict(test_kind=2, test_M=1e10, test_a=1.0))
    x = _points(100, 12, Rmax=3.0, zmax=3.0)
    lap = (4 * _laplacian(orc, pot, x, orc.TEST, 1e-3) - _laplacian(orc, pot, x, orc.TEST, 2e-3)) / 3
    rho = orc.density(pot, x, orc.TEST)
    np.testing.assert_allclose(lap, 4 * np.pi * G * rho, rtol=1e-6)


@pytest.mark.parametrize("mask_name", ["DISC", "HALO", "BAR", "ALL"])
def test_force_is_minus_gradient(orc, mask_name):
    pot = _pot(orc)
    mask = (orc.DISC | orc.HALO | orc.BAR) if mask_name == "ALL" else getattr(orc, mask_name)
    x = np.concatenate([_points(300, 13), _points(50, 14, Rmax=30.0, zmax=10.0),
                        np.array([[4.0, 0.0, 0.0], [-4.0, 0.1, 0.0], [12.0, -3.0, 0.5], [-30.0, 2.0, -1.0]])])
    _, acc = orc.potential(pot, x, mask)
    h = 1e-5
    for k in range(3):
        e = np.zeros(3); e[k] = h
        pp, _ = orc.potential(pot, x + e, mask)
        pm, _ = orc.potential(pot, x - e, mask)
        fd = -(pp - pm) / (2 * h)
        scale = np.linalg.norm(acc, axis=1)
        assert np.all(np.abs(fd - acc[:, k]) <= 1e-6 * scale + 1e-14)


def test_bar_equals_needle_quadrature_of_mn(orc):
    """Eq. Rn_to_In with n = 1, eta = 0: the closed-form bar potential equals
    the average of MN potentials over the needle x' in [-L, L]."""
    p = dict(bar_M=1e10, bar_L=4.0, bar_b=1.0, bar_c=0.5)
    bar = orc.make_pot(p)
    mn = orc.make_pot(dict(disc_M=p["bar_M"], disc_a=p["bar_b"], disc_b=p["bar_c"]))
    x = np.concatenate([_points(40, 15, Rmax=10, zmax=2), np.array([[3.9, 0.0, 0.0], [-20.0, 1.0, 1.0]])])
    phi_bar, acc_bar = orc.potential(bar, x, orc.BAR)
    gx, gw = leggauss(200)
    L = p["bar_L"]
    s = L * gx
    phi_q = np.zeros(len(x)); acc_q = np.zeros((len(x), 3))
    for sj, wj in zip(s, gw):
        ph, ac = orc.potential(mn, x - np.array([sj, 0, 0]), orc.DISC)
        phi_q += wj * ph / 2.0
        acc_q += wj * ac / 2.0
    np.testing.assert_allclose(phi_bar, phi_q, rtol=1e-12)
    np.testing.assert_allclose(acc_bar, acc_q, rtol=1e-9, atol=1e-12 * np.abs(acc_bar).max())


def test_bar_short_needle_limit_is_mn(orc):
    x = _points(30, 16)
    mn = orc.make_pot(dict(disc_M=1e10, disc_a=1.0, disc_b=0.5))
    bar = orc.make_pot(dict(bar_M=1e10, bar_L=1e-5, bar_b=1.0, bar_c=0.5))
    p1, a1 = orc.potential(mn, x, orc.DISC)
    p2, a2 = orc.potential(bar, x, orc.BAR)
    np.testing.assert_allclose(p2, p1, rtol=1e-8)
    np.testing.assert_allclose(a2, a1, rtol=1e-6, atol=1e-9 * np.abs(a1).max())


def test_nfw_reparameterisation(orc):
    """Sec. 3.2.1: with Delta = 200, M(<R_vir) must equal M_vir, and
    R_vir^3 = 3 M_vir / (4 pi 200 rho_crit)."""
    for M200, c, H0 in [(1e12, 10.0, 70.0), (5e11, 5.0, 67.7), (2e12, 20.0, 70.0)]:
        Mdm, rs = orc.nfw_from_m200(M200, c, H0)
        Rv = c * rs
        assert orc.nfw_enclosed(Mdm, rs, Rv) == pytest.approx(M200, rel=1e-13)
        H = H0 / 1000.0
        rho_c = 3 * H * H / (8 * math.pi * G)
        assert 4.0 / 3.0 * math.pi * Rv ** 3 * 200 * rho_c == pytest.approx(M200, rel=1e-12)


def test_nfw_enclosed_mass_matches_density_integral(orc):
    pot = orc.make_pot(dict(halo_M200=1e12, halo_c=10.0, H0=70.0))
    Mdm, rs = pot.halo_Mdm, pot.halo_rs
    gx, gw = leggauss(400)
    for R in [0.5, 5.0, 30.0, 200.0]:
        # integrate 4 pi r^2 rho(r) dr with r = R u^2 (smooths the r^-1 cusp)
        u = 0.5 * (gx + 1)
        r = R * u * u
        rho = orc.density(pot, np.stack([r, 0 * r, 0 * r], 1), orc.HALO)
        m = np.sum(0.5 * gw * 4 * math.pi * r * r * rho * 2 * R * u)
        assert m == pytest.approx(orc.nfw_enclosed(Mdm, rs, R), rel=1e-10)


def test_nfw_centre_is_finite(orc):
    pot = orc.make_pot(dict(halo_M200=1e12, halo_c=10.0, H0=70.0))
    x = np.array([[1e-9, 0, 0], [1e-6, 1e-6, 0], [1e-3, 0, 0]])
    phi, acc = orc.potential(pot, x, orc.HALO)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(acc))
    # |a| -> G M_DM / (2 R_s^2) at the centre
    lim = G * pot.halo_Mdm / (2 * pot.halo_rs ** 2)
    assert np.linalg.norm(acc[0]) == pytest.approx(lim, rel=1e-6)
