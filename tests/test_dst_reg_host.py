"""The register-resident DST-I and DCT-I phases of the float32 transform
kernels, run on the host one simulated thread at a time, against scipy's
DST-I / DCT-I: checks the two-level index decomposition, the exchange layout,
the split pairing, the first odd output of the cosine transform and the
segmented scan for every tile length the kernels use (no GPU needed)."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.fft

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_05024_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("dstreg") / "dst_reg_host")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fno-strict-aliasing", "-I", CSRC,
                    os.path.join(HERE, "host", "dst_reg_host.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("N", [32, 64, 128, 256, 384, 512])
@pytest.mark.parametrize("RS", [32, 33])
def test_register_dst_matches_scipy(harness, N, RS):
    x = np.random.default_rng(N + RS).standard_normal((32, N - 1))
    inp = f"{N} {RS} 0\n" + "\n".join(" ".join(f"{v:.9g}" for v in row) for row in x)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout
    y = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    ref = scipy.fft.dst(x, type=1, axis=1) / 2.0     # sum_j x_j sin(pi j k / N)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("N", [32, 64, 128, 256, 384, 512])
@pytest.mark.parametrize("RS", [32, 33])
def test_register_dct_matches_scipy(harness, N, RS):
    x = np.random.default_rng(2 * N + RS).standard_normal((32, N + 1))
    inp = f"{N} {RS} 1\n" + "\n".join(" ".join(f"{v:.9g}" for v in row) for row in x)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout
    y = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    ref = scipy.fft.dct(x, type=1, axis=1) / 2.0     # sum_j c_j x_j cos(pi j k / N)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err
