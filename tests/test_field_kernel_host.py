"""The force-field device functions of k_orbit.cu (the per-orbit part shared by every
orbit kernel) compiled for the host in both precisions and compared with the oracle's
potential and acceleration: the paper's Dehnen-Aly bar (Sec. 2.1.2, App. A; bar_kind 1:
T3 long bar by the closed-form needle integrals, V4 bulge by 8-point Gauss-Legendre
quadrature) on top of the disc and halo, and the Long-Murali bar as a control.  This
checks the kernel's arithmetic on the CPU; the GPU runs it in tests/test_gpu_orbit.py."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2607_00117_gb300 import inputs
from test_bs3_kernel_host import CSRC, CUDA_INC, HERE, SHIMS

PAPER_BAR = dict(inputs.DISC_HALO, bar_M=1e10, bar_L=4.0, bar_kind=1)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = open(os.path.join(CSRC, "k_orbit.cu")).read()
    a = src.index("// ---- precision-dispatched math")
    b = src.index("// ---- end of the per-orbit device functions")
    body = src[a:b].replace("__device__ __forceinline__", "inline").replace("__device__", "")
    d = tmp_path_factory.mktemp("fieldhost")
    (d / "bs3_host.h").write_text(SHIMS + "inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }\n" + body +
                                  "\n}  // namespace sw\n")
    exe = d / "field_host"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", f"-I{d}", f"-I{CSRC}", f"-I{CUDA_INC}",
           os.path.join(HERE, "host_harness", "field_main.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def _points(seed, n):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(0, 3, (n // 2, 3)), rng.normal(0, 12, (n - n // 2 - 6, 3)),
                           np.array([[0.0, 0, 0], [4.0, 0, 0], [-4.0, 0.01, 0], [0.05, 0, 0.02],
                                     [30.0, -20.0, 5.0], [1e-4, 1e-4, 0]])])


def _run(harness, orc, p, xyz):
    exe, d = harness
    Mdm, rs = orc.nfw_from_m200(p["halo_M200"], p["halo_c"], p.get("H0", 70.0))
    P = [p["disc_M"], p["disc_a"], p["disc_b"], Mdm, rs, p.get("bar_M", 0.0), p.get("bar_L", 1.0),
         p.get("bar_b", 1.0), p.get("bar_c", 1.0), p.get("bar_kind", 0)]
    x, w = np.polynomial.legendre.leggauss(8)
    gl = np.concatenate([x[4:][::-1], w[4:][::-1]])
    fin, fout = d / "in.bin", d / "out.bin"
    with open(fin, "wb") as f:
        np.array(P + list(gl) + [len(xyz)], dtype=np.float64).tofile(f)
        np.ascontiguousarray(xyz, dtype=np.float64).tofile(f)
    subprocess.run([str(exe), str(fin), str(fout)], check=True)
    raw = np.fromfile(fout, dtype=np.float64)
    n = len(xyz)
    out = []
    for k in range(3):
        blk = raw[4 * n * k:4 * n * (k + 1)]
        out.append((blk[:n], blk[n:].reshape(n, 3)))
    return out


@pytest.mark.parametrize("pot", ["paper_bar", "long_murali"])
def test_field_device_functions_match_oracle(orc, harness, pot):
    p = PAPER_BAR if pot == "paper_bar" else dict(inputs.DISC_HALO, **inputs.BAR)
    xyz = _points(301, 1000)
    phi_o, acc_o = orc.potential(orc.make_pot(p), xyz)
    (phi64, acc64), (phi32, acc32), (phid, accd) = _run(harness, orc, p, xyz)
    scale = _scale(acc_o)
    np.testing.assert_allclose(phi64, phi_o, rtol=1e-11)
    assert np.all(np.abs(acc64 - acc_o) <= 1e-12 * scale), (np.abs(acc64 - acc_o) / scale).max()
    # FP32, and the fixed disc + halo + Long-Murali layout of the FP32 kernels (its branch-free forms)
    for ph, ac in ((phi32, acc32), (phid, accd)):
        np.testing.assert_allclose(ph, phi_o, rtol=1e-6)
        assert np.all(np.abs(ac - acc_o) <= 3e-5 * scale), (np.abs(ac - acc_o) / scale).max()


def _scale(acc):
    """|a| per point, floored at 1e-3 of the sample's median |a| (at the centre the
    force vanishes by symmetry and only an absolute error is meaningful)."""
    n = np.linalg.norm(acc, axis=1, keepdims=True)
    return np.maximum(n, 1e-3 * np.median(n))


def test_paper_bar_part_alone(orc, harness):
    """The bar's own potential and force (disc and halo off), where a wrong coefficient or
    sign of the T3 or V4 terms is not hidden under the axisymmetric part."""
    p = dict(disc_M=0.0, disc_a=3.0, disc_b=0.3, halo_M200=0.0, halo_c=10.0, bar_M=1e10, bar_L=4.0, bar_kind=1)
    xyz = _points(302, 600)
    phi_o, acc_o = orc.potential(orc.make_pot(p), xyz, mask=orc.BAR)
    (phi64, acc64), (phi32, acc32) = _run_bar_only(harness, orc, p, xyz)
    scale = _scale(acc_o)
    np.testing.assert_allclose(phi64, phi_o, rtol=1e-12)
    assert np.all(np.abs(acc64 - acc_o) <= 1e-11 * scale), (np.abs(acc64 - acc_o) / scale).max()
    # FP32: the closed forms' differences of antiderivatives lose digits far from the needle
    np.testing.assert_allclose(phi32, phi_o, rtol=3e-5)
    assert np.all(np.abs(acc32 - acc_o) <= 1e-4 * scale), (np.abs(acc32 - acc_o) / scale).max()


def _run_bar_only(harness, orc, p, xyz):
    exe, d = harness
    P = [0.0, p["disc_a"], p["disc_b"], 0.0, 1.0, p["bar_M"], p["bar_L"], 1.0, 1.0, 1]
    x, w = np.polynomial.legendre.leggauss(8)
    gl = np.concatenate([x[4:][::-1], w[4:][::-1]])
    fin, fout = d / "in2.bin", d / "out2.bin"
    with open(fin, "wb") as f:
        np.array(P + list(gl) + [len(xyz)], dtype=np.float64).tofile(f)
        np.ascontiguousarray(xyz, dtype=np.float64).tofile(f)
    subprocess.run([str(exe), str(fin), str(fout)], check=True)
    raw = np.fromfile(fout, dtype=np.float64)
    n = len(xyz)
    return [(raw[4 * n * k:4 * n * k + n], raw[4 * n * k + n:4 * n * (k + 1)].reshape(n, 3)) for k in range(2)]
