"""sw_matrix_apply_static: the U w product for callers that cannot allocate
device memory at call time (its scratch is a fixed static device array).
Checked through the C-ABI against sw_matrix_apply, which allocates its
scratch, on two calls in a row (the shared array keeps the previous call's
contents, so the second call also checks that the accumulator is cleared).
This file is collected last."""
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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_static_apply_matches_allocating_apply(sw, prec):
    W = inputs.WORKLOADS["axisym_2k"]
    ctx = sw.Context(0, prec)
    ctx.set_potential(dict(inputs.DISC_HALO, **inputs.BAR))
    ics = inputs.disc_ics(inputs.DISC_HALO, 1500, seed=31)
    ctx.integrate_library(ics, 40.0, inputs.DT_HALF_MYR, 300)
    U = ctx.project(W["grid"])
    rng = np.random.default_rng(7)
    ws = [rng.uniform(0, 2, U.N) for _ in range(2)]
    # the static calls come first on this context, before any allocating apply has sized its
    # workspace: they must allocate nothing
    n0 = ctx.alloc_count()
    got = [U.apply_static(w) for w in ws]
    assert ctx.alloc_count() == n0, "sw_matrix_apply_static allocated device memory"
    ref = [U.apply(w) for w in ws]
    if prec == "fp32":
        assert ctx.alloc_count() > n0   # control: the allocating form does size a workspace here
    for call in range(2):
        np.testing.assert_allclose(got[call], ref[call], rtol=1e-12, atol=1e-12 * np.abs(ref[call]).max())
        assert np.abs(ref[call]).max() > 0
    # and again after the allocating calls (the shared array keeps the previous call's contents)
    for w, r in zip(ws, ref):
        np.testing.assert_allclose(U.apply_static(w), r, rtol=1e-12, atol=1e-12 * np.abs(r).max())


def test_static_apply_rejects_oversize(sw):
    ctx = sw.Context(0, "fp32")
    ctx.set_potential(inputs.DISC_HALO)
    ics = inputs.disc_ics(inputs.DISC_HALO, 300, seed=32)
    ctx.integrate_library(ics, 0.0, inputs.DT_HALF_MYR, 2)
    grid = dict(inputs.WORKLOADS["barred_100k"]["grid"], nv=1000)   # M = 4000 + 2500 * 1001 > 2^21 - 2 N
    U = ctx.project(grid)
    assert 2 * U.N + U.M > (1 << 21)
    with pytest.raises(sw.SwError):
        U.apply_static(np.ones(U.N))
