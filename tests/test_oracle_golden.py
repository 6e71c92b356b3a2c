"""The oracle's run of Algorithm 2 (O2) reaches the exact eigenvalues of the oracle's
dense solve (O1) stored under tests/golden/, and the FFT stage code used by the CUDA
kernels is checked on the host against a direct DFT."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import chebyshev as ch
from oracle.planewave import PWOperator
from synth import config_cell

HERE = os.path.dirname(os.path.abspath(__file__))


def test_golden_file_is_the_dense_spectrum_of_nc24():
    cell = config_cell("nc24")
    gold = np.loadtxt(os.path.join(HERE, "golden", "nc24_exact_eigs.txt"))
    assert gold.shape == (48,)
    assert np.all(np.diff(gold) >= 0)
    # the lowest eigenvalue is below the lowest potential well's floor plus kinetic zero
    assert gold[0] > cell.vloc.min() - 1.0


def test_algorithm2_reaches_exact_eigenvalues_nc24():
    """nc24: degree 8, lambda_+ = E_cut bound; lowest 24 of 32 within 1e-8 Ha.  From the
    random start 5 sweeps leave 5.5e-7 Ha; 7 sweeps give 2.5e-10 Ha."""
    cell = config_cell("nc24")
    gold = np.loadtxt(os.path.join(HERE, "golden", "nc24_exact_eigs.txt"))
    op = PWOperator.from_cell(cell)
    res = ch.solve(op, cell.Y0, degree=8, sweeps=7, mode="paper")
    assert np.abs(res["w"][:24] - gold[:24]).max() <= 1e-8
    assert np.all(res["w"] >= gold[:32] - 1e-10)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_fft_stage_code_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(HERE, "native", "fft_core_check.cu")
    exe = str(tmp_path / "fftcheck")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(float, l.split())) for l in out if l.strip()]
    assert len(rows) >= 30
    for n, d64a, d64b, d32a, d32b in rows:
        assert d64a < 2e-15 and d64b < 2e-15, n
        assert d32a < 1e-6 and d32b < 1e-6, n


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_two_pass_fft_code_on_host(tmp_path):
    """The compile-time-length line FFTs (split-order F and its transpose G) against a
    direct DFT, run pass by pass on the host."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(HERE, "native", "fft_fast_check.cu")
    exe = str(tmp_path / "fftfast")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(float, l.split())) for l in out if l.strip()]
    assert [int(r[0]) for r in rows] == [16, 24, 32, 48, 64, 72, 96, 120, 128, 144]
    for n, f64, g64, f32, g32 in rows:
        assert f64 < 2e-15 and g64 < 2e-15, n
        assert f32 < 1e-6 and g32 < 1e-6, n
