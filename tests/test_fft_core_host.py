"""The CUDA path's batched-FFT pieces (radix DFTs, Stockham pass indexing, pass-twiddle
exponents, shared-memory padding), compiled for the host and run thread by thread in the
order the kernel's barriers impose, against a direct DFT in double precision."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_core_host")
    src = os.path.join(ROOT, "tests", "host", "fft_core_host.cu")
    inc = os.path.join(ROOT, "paper_2506_18003_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-I", inc,
                    "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {int(a): float(b) for a, b in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("M", [2 ** e for e in range(1, 15)])
def test_fft_size(results, M):
    assert results[M] < 2e-6, results[M]
