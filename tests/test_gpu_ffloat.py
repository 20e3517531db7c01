"""Float-pair helpers of the epilogues (csrc/ffloat.cuh) against FP64 on the GPU.

The half-step epilogues compute the mass terms of the TI update through a
table-driven exp2 on float pairs; its relative error must stay far below the
1e-9 the translation of Prop. 2 needs.  Products and sums of pairs must agree
with FP64 to ~2^-44, and the pair log that finalises the mass sums with
FP64's to within exp2's relative error (its Newton step evaluates 2^-y0 with it).
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_ffloat_accuracy(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "ffloat_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "paper_2201_00730_gb300", "csrc"),
                    os.path.join(HERE, "cuda", "ffloat_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = dict(zip(out[0::2], map(float, out[1::2])))
    assert vals["exp2"] < 1e-11, vals
    assert vals["mul"] < 2.0 ** -43, vals
    assert vals["add"] < 2.0 ** -43, vals
    assert vals["log"] < 1e-11, vals


def test_mass_reduction_against_fp64(tmp_path):
    """The TI half-step's mass reduction <w, e^{-v/rho}> (Prop. 2's log-ratio takes its log) as the
    fused epilogues compute it on float pairs, over 262144 terms (the largest workload's size) and
    with term ranges up to 2^+-87, against the same sum in long double: relative error below 1e-10,
    i.e. far below the FP32 rounding (6e-8) of the potentials that feed it."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "mass_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "paper_2201_00730_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "cuda", "mass_check.cu"), "-o", exe], check=True)
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.strip().splitlines()
    assert len(lines) == 4, lines
    for line in lines:
        f = line.split()
        vals = dict(zip(f[0::2], f[1::2]))
        assert int(vals["status"]) == 0, line
        assert float(vals["relerr"]) < 1e-10, line
