"""The adaptive integrator's device functions (k_orbit.cu, the per-orbit part of the
Bogacki-Shampine path) compiled for the host in their FP64 form and compared with
the oracle's build_matrix_bs3 (Sec. 2.2.2, Sec. 2.2.4): same step sequence, same
integration times and the same step-weighted columns to rounding.  This checks the
kernel's arithmetic on the CPU; its launch on the GPU is a separate test."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2607_00117_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

SHIMS = """// host stand-ins for the device intrinsics the per-orbit functions use
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include "sw_common.cuh"
using std::fmax; using std::fmin; using std::isfinite;
inline float __frsqrt_rn(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float __fdiv_rn(float a, float b) { return a / b; }
inline float __expf(float x) { return std::exp(x); }
// rounding-down conversion, saturating like the device instruction (NaN gives 0)
inline int __float2int_rd(float x) {
    if (!(x == x)) return 0;
    const double f = std::floor((double)x);
    return f >= 2147483647.0 ? INT32_MAX : (f <= -2147483648.0 ? INT32_MIN : (int)f);
}
template <class T> inline T atomicAdd(T* p, T v) { T o = *p; *p = o + v; return o; }
template <class T> inline T atomicMax(T* p, T v) { T o = *p; if (v > o) *p = v; return o; }
inline long long __double_as_longlong(double d) { long long r; std::memcpy(&r, &d, 8); return r; }
inline unsigned __ballot_sync(unsigned, bool b) { return b ? 1u : 0u; }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
template <class T> inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
struct HostIdx { unsigned x = 0; };
static HostIdx threadIdx;
namespace sw {
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = open(os.path.join(CSRC, "k_orbit.cu")).read()
    a = src.index("// ---- precision-dispatched math")
    b = src.index("// ---- end of the per-orbit device functions")
    body = src[a:b].replace("__device__ __forceinline__", "inline").replace("__device__", "")
    d = tmp_path_factory.mktemp("bs3host")
    (d / "bs3_host.h").write_text(SHIMS + body + "\n}  // namespace sw\n")
    exe = d / "bs3_host"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", f"-I{d}", f"-I{CSRC}", f"-I{CUDA_INC}",
           os.path.join(HERE, "host_harness", "bs3_main.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def _run(harness, p, Mdm, rs, omega, grid, ics, S, rtol, gh_v0s=None):
    exe, d = harness
    P = [p["disc_M"], p["disc_a"], p["disc_b"], Mdm, rs, p.get("bar_M", 0.0), p.get("bar_L", 1.0),
         p.get("bar_b", 1.0), p.get("bar_c", 1.0), omega, grid["incl"], grid.get("bar_angle", 0.0),
         inputs.DT_HALF_MYR, rtol, S, len(ics)]
    G = [grid["nx"], grid["ny"], grid["pix"], grid["nv"], grid["vmax"], grid["nR"], grid["nphi"], grid["nz"],
         grid.get("Rmax", 10.0), grid.get("zmin", -3.0), grid.get("zmax", 3.0), 1.0 if gh_v0s is not None else 0.0]
    fin, fout = d / "in.bin", d / "out.bin"
    with open(fin, "wb") as f:
        np.array(P + G, dtype=np.float64).tofile(f)
        np.ascontiguousarray(ics, dtype=np.float64).tofile(f)
        if gh_v0s is not None:
            np.ascontiguousarray(gh_v0s, dtype=np.float64).tofile(f)
    subprocess.run([str(exe), str(fin), str(fout)], check=True)
    return np.fromfile(fout, dtype=np.float64)


@pytest.mark.parametrize("barred", [True, False])
def test_bs3_device_functions_match_oracle(orc, harness, barred):
    p = dict(inputs.DISC_HALO, **inputs.BAR) if barred else dict(inputs.DISC_HALO)
    omega = 40.0 if barred else 0.0
    Mdm, rs = orc.nfw_from_m200(p["halo_M200"], p["halo_c"], p.get("H0", 70.0))
    grid = dict(inputs.WORKLOADS["barred_100k"]["grid"])
    grid.update(nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    S, rtol = 500, 1e-4
    ics = inputs.disc_ics(inputs.DISC_HALO, 40, seed=131)
    raw = _run(harness, p, Mdm, rs, omega, grid, ics, S, rtol)
    obs = orc.make_obs(grid)
    M = orc.n_rows(obs)
    Uh, th = raw[:M * len(ics)].reshape(len(ics), M), raw[M * len(ics):]
    opts = orc.bs3_opts(rtol=rtol, h0=inputs.DT_HALF_MYR)
    Uo, _, so = orc.build_matrix_bs3(orc.make_pot(p), omega, opts, S, ics, obs)
    assert np.all(so == 0)
    t_o = np.array([orc.bs3_trajectory(orc.make_pot(p), omega, opts, S, ic)[0][-1] for ic in ics])
    np.testing.assert_allclose(th, t_o, rtol=1e-10)
    assert np.abs(Uh - Uo).sum(1).max() < 1e-9
    np.testing.assert_allclose(Uh[:, :500].sum(1), Uo[:, :500].sum(1), rtol=1e-10)


def test_bs3_device_functions_gauss_hermite_rows(orc, harness):
    """The same check with Gauss-Hermite rows: each copy in pixel p adds its step weight
    times 2 sqrt(pi) alpha(w) H_m(w), w = (V - v0_p) / s_p."""
    p = dict(inputs.DISC_HALO, **inputs.BAR)
    Mdm, rs = orc.nfw_from_m200(p["halo_M200"], p["halo_c"], p.get("H0", 70.0))
    grid = dict(inputs.WORKLOADS["barred_100k"]["grid"])
    grid.update(nx=12, ny=10, nv=1, nR=6, nphi=8, nz=4, gh=1)
    rng = np.random.default_rng(6)
    v0s = np.stack([rng.normal(0, 40, 120), rng.uniform(60, 160, 120)], 1)
    S = 400
    ics = inputs.disc_ics(inputs.DISC_HALO, 30, seed=107)
    raw = _run(harness, p, Mdm, rs, 40.0, grid, ics, S, 1e-4, gh_v0s=v0s)
    obs = orc.make_obs(grid)
    M = orc.n_rows(obs)
    Uh = raw[:M * len(ics)].reshape(len(ics), M)
    Uo, _, so = orc.build_matrix_bs3(orc.make_pot(p), 40.0, orc.bs3_opts(rtol=1e-4, h0=inputs.DT_HALF_MYR), S, ics,
                                     obs, gh_v0s=v0s)
    assert np.all(so == 0)
    np.testing.assert_allclose(Uh, Uo, rtol=1e-9, atol=1e-12)
