"""Host-side check of the persistent schedule's task builder (no GPU): the
fast, multi-threaded builder against the reference replay of the phases, on
seeded random layouts (1-4 levels, ragged sizes, periodic or not, 1-3 coarse
steps per list) -- same tasks, edges a backwards subset of the reference,
identical transitive closures, identical lists on 1 and 4 threads."""
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
    out = os.path.join(tempfile.mkdtemp(prefix="vlbm_tasks_"), "task_builder_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-I", os.path.join(ROOT, "paper_2609_35529_b300", "csrc"),
                    os.path.join(ROOT, "tests", "task_builder_check.cpp"), "-o", out], check=True)
    return out


@pytest.mark.parametrize("seed", [7, 2026])
def test_fast_builder_orders_tasks_like_the_reference(checker, seed):
    r = subprocess.run([checker, "--layouts", "200", "--seed", str(seed)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK"), r.stdout
