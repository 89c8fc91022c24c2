"""Host-side logic that needs no GPU: the dithered orbit bundles' initial
conditions and the benchmark's roofline arithmetic."""
import math

import numpy as np

from paper_2607_00117_gb300 import inputs


def test_dither_draws_bundles_inside_the_box():
    """Orbit bundles (Sec. 2.2.1): n realisations per initial condition, consecutive,
    each inside a box 0.1 kpc wide in position and 5% of v_c wide in velocity,
    centred on the initial condition; reproducible from the seed."""
    p = inputs.WORKLOADS["barred_100k"]["potential"]
    base = inputs.disc_ics(p, 50, seed=7)
    d = inputs.dither(base, 4, 8, p)
    assert d.shape == (200, 6)
    np.testing.assert_array_equal(d, inputs.dither(base, 4, 8, p))
    off = d - np.repeat(base, 4, axis=0)
    assert np.all(np.abs(off[:, :3]) <= 0.05 + 1e-12)
    vc = inputs._vcirc(np.hypot(base[:, 0], base[:, 1]), base[:, 2], p)
    assert np.all(np.abs(off[:, 3:]) <= 0.025 * np.repeat(vc, 4)[:, None] + 1e-12)
    # the realisations of one bundle differ and are centred on average
    assert np.all(np.abs(off).sum(axis=1) > 0)
    assert abs(off[:, 0].mean()) < 0.01


def test_roofline_entry_arithmetic():
    import bench
    stats = {
        "k_bytes": {"launches": 2, "ms": 4.0, "work": 2 * 6.0e9, "kind": "bytes"},
        "k_tensor": {"launches": 1, "ms": 1.0, "work": 1.0e12, "kind": "flop_tensor"},
        "k_simt": {"launches": 4, "ms": 8.0, "work": 4 * 4.0e10, "kind": "flop_simt"},
        "k_orbit": {"launches": 1, "ms": 100.0, "work": 1.0e9, "kind": "orbit_steps"},
    }
    r = bench.roofline_entry("k_bytes", stats, 6000.0, 1700.0, 2070.0, 152)
    assert r["bound"] == "hbm" and math.isclose(r["achieved"], 3000.0) and math.isclose(r["frac"], 0.5)
    r = bench.roofline_entry("k_tensor", stats, 6000.0, 1700.0, 2070.0, 152)
    assert r["bound"] == "tensor" and math.isclose(r["achieved"], 1000.0)
    r = bench.roofline_entry("k_simt", stats, 6000.0, 1700.0, 2070.0, 152)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["bound"] == "alu" and math.isclose(r["achieved"], 20.0) and math.isclose(r["peak"], peak)
    assert "one_sm_frac" not in r
    one = {"diag_factor_inverse": {"launches": 10, "ms": 0.5, "work": 10 * 1.0e5, "kind": "flop_simt"}}
    r = bench.roofline_entry("diag_factor_inverse", one, 6000.0, 1700.0, 2070.0, 152)
    assert math.isclose(r["achieved"], 2e-3) and math.isclose(r["one_sm_frac"], r["frac"] * 152)
    r = bench.roofline_entry("k_orbit", stats, 6000.0, 1700.0, 2070.0, 152)
    assert math.isclose(r["achieved"], bench.OPS_PER_ORBIT_STEP * 1e9 / 0.1 / 1e12)
    assert math.isclose(r["peak"], 152 * 128 * 2070e6 / 1e12)
    assert math.isclose(r["algorithmic_frac"], bench.ALG_OPS_PER_ORBIT_STEP * 1e9 / 0.1 / 1e12 / r["peak"])
    # split products: the Gram counts the three issued, the factor updates the method's one
    st3 = {"gram_tcgen05": {"launches": 1, "ms": 1.0, "work": 1.5e12, "kind": "flop_tensor"},
           "syrk_update_tcgen05": {"launches": 1, "ms": 1.0, "work": 0.5e12, "kind": "flop_tensor"}}
    g = bench.roofline_entry("gram_tcgen05", st3, 6000.0, 1500.0, 2070.0, 152)
    assert math.isclose(g["frac"], 1.0) and math.isclose(g["method_frac"], 1.0 / 3.0)
    y = bench.roofline_entry("syrk_update_tcgen05", st3, 6000.0, 1500.0, 2070.0, 152)
    assert math.isclose(y["frac"], 1.0 / 3.0) and math.isclose(y["tensor_pipe_frac"], 1.0)


def test_reference_arm_reports_the_workload_rows(orc):
    """The reference arm's config is the workload's: its row counts are those of the oracle's
    observation grids (the histogram matrix, and the Gauss-Hermite rows the solve uses)."""
    import bench
    W = inputs.WORKLOADS[bench.WORKLOAD]
    c = bench.reference_config(W, 1)
    assert c["rows_histogram"] == orc.n_rows(orc.make_obs(W["grid"]))
    assert c["rows_solve"] == orc.n_rows(orc.make_obs(dict(W["grid"], gh=1)))
    assert c["bundles"] * c["dithers_per_bundle"] == c["n_orb"] == W["n_orb"]
    assert c["parallelism"] == "replicas x1"
