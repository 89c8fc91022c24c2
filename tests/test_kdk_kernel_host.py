"""The kick-drift-kick orbit body of k_orbit.cu (the benchmark's per-orbit path: force, Kahan-compensated
step in FP32, bar frame, the four mirror copies of Table 1, the z-x-z projection and the run-length binning
into integer counts, Sec. 2.2.2-2.2.4) compiled for the host and compared with the oracle's build_matrix:
the FP64 form's counts bit-exact over 64 steps, and the FP32 form (the fixed disc + halo + Long-Murali layout
of the FP32 kernels for the barred model) moving at most a few samples across bin edges.  This checks the
kernel's arithmetic and its branch-free bookkeeping on the CPU; the GPU runs them in tests/test_gpu_orbit.py."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs
from test_bs3_kernel_host import CSRC, CUDA_INC, HERE, SHIMS


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = open(os.path.join(CSRC, "k_orbit.cu")).read()
    a = src.index("// ---- precision-dispatched math")
    b = src.index("// ---- end of the per-orbit device functions")
    body = src[a:b].replace("__device__ __forceinline__", "inline").replace("__device__", "")
    d = tmp_path_factory.mktemp("kdkhost")
    (d / "bs3_host.h").write_text(SHIMS + body + "\n}  // namespace sw\n")
    exe = d / "kdk_host"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", f"-I{d}", f"-I{CSRC}", f"-I{CUDA_INC}",
           os.path.join(HERE, "host_harness", "kdk_main.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def _run(harness, p, Mdm, rs, omega, grid, ics, S):
    exe, d = harness
    P = [p["disc_M"], p["disc_a"], p["disc_b"], Mdm, rs, p.get("bar_M", 0.0), p.get("bar_L", 1.0),
         p.get("bar_b", 1.0), p.get("bar_c", 1.0), omega, grid["incl"], grid.get("bar_angle", 0.0),
         inputs.DT_HALF_MYR, 0.0, S, len(ics)]
    G = [grid["nx"], grid["ny"], grid["pix"], grid["nv"], grid["vmax"], grid["nR"], grid["nphi"], grid["nz"],
         grid.get("Rmax", 10.0), grid.get("zmin", -3.0), grid.get("zmax", 3.0), 0.0]
    fin, fout = d / "in.bin", d / "out.bin"
    with open(fin, "wb") as f:
        np.array(P + G, dtype=np.float64).tofile(f)
        np.ascontiguousarray(ics, dtype=np.float64).tofile(f)
    subprocess.run([str(exe), str(fin), str(fout)], check=True)
    raw = np.fromfile(fout, dtype=np.float64)
    return raw[:len(raw) // 2], raw[len(raw) // 2:]


@pytest.mark.parametrize("barred", [True, False])
def test_kdk_orbit_body_matches_oracle(orc, harness, barred):
    p = dict(inputs.DISC_HALO, **inputs.BAR) if barred else dict(inputs.DISC_HALO)
    omega = 40.0 if barred else 0.0
    Mdm, rs = orc.nfw_from_m200(p["halo_M200"], p["halo_c"], p.get("H0", 70.0))
    grid = dict(inputs.WORKLOADS["barred_100k"]["grid"], bar_angle=0.5)
    grid.update(nx=20, ny=20, nv=16, nR=10, nphi=10, nz=5)
    S = 64
    ics = inputs.disc_ics(inputs.DISC_HALO, 60, seed=141)
    u64, u32 = _run(harness, p, Mdm, rs, omega, grid, ics, S)
    obs = orc.make_obs(grid)
    M = orc.n_rows(obs)
    n = len(ics)
    Uo, _, so = orc.build_matrix(orc.make_pot(p), omega, inputs.DT_HALF_MYR, S, ics, obs)
    assert np.all(so == 0)
    c_o = np.rint(Uo * 4 * S)
    c64 = np.rint(u64.reshape(n, M) * 4 * S)
    c32 = np.rint(u32.reshape(n, M) * 4 * S)
    # FP64: every sample of every copy in the same density cell, pixel and velocity bin as the oracle's
    np.testing.assert_array_equal(c64, c_o)
    # FP32: the same total per row kind; a sample within rounding of a bin edge may land in the neighbour
    # (each such sample-copy moves one count: an L1 difference of two)
    assert np.array_equal(c32.sum(1), c_o.sum(1))
    moved = np.abs(c32 - c_o).sum() / 2
    total = c_o.sum()
    assert moved <= 2e-3 * total, (moved, total)
