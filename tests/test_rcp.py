"""The integer-pipe reciprocal used by the collision (rcp_rn.cuh) gives the
IEEE division 1.0 / x bit for bit: on the host (no GPU) with the FP32
division seed and seeds perturbed by up to 3 * 2^-21 relative, over seeded
random doubles of every kind plus every power of two and its neighbours;
on the GPU with the device seed (FP32 reciprocal approximation)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = os.path.join(tempfile.mkdtemp(prefix="vlbm_rcp_"), "rcp_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2609_35529_b300", "csrc"),
                    os.path.join(ROOT, "tests", "rcp_check.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("seed", [5, 2026])
def test_reciprocal_is_the_ieee_division_on_the_host(checker, seed):
    r = subprocess.run([checker, "--n", "3000000", "--seed", str(seed)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK"), r.stdout


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [1, 2])
def test_reciprocal_is_the_ieee_division_on_the_gpu(seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm
    build.build()
    bad, unsettled, first = vlbm.selftest_rcp(seed, 1 << 28)
    assert bad == 0 and unsettled == 0, (bad, unsettled, first)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [1, 2])
def test_division_is_the_ieee_division_on_the_gpu(seed):
    """The sensor's quotients (integer-pipe reciprocal, then two remainder
    corrections) are the FP64 division's bits on 2^28 seeded pairs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm
    build.build()
    bad, first = vlbm.selftest_div(seed, 1 << 28)
    assert bad == 0, (bad, first)
