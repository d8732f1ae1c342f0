"""The host planner (plan.cpp) and the job-image builder (program.cpp) under AddressSanitizer
and UBSan: tests/sanitize/planner_driver.cpp builds transform plans over a sweep of ring sizes,
lengths, weights and both omega modes, and job images of every single-CTA and cluster shape.
An out-of-bounds access or undefined behaviour on the host side of the path fails the run.
CPU only; skipped where the compiler has no sanitizer runtimes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0810_3203_gb300", "csrc")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.mark.slow
def test_planner_under_address_and_ub_sanitizers(tmp_path):
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path / "planner_driver")
    cmd = [cxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
           "-fno-omit-frame-pointer", "-I" + os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "sanitize", "planner_driver.cpp"), os.path.join(CSRC, "plan.cpp"),
           os.path.join(CSRC, "program.cpp"), "-L" + os.path.join(CUDA, "lib64"), "-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "asan" in r.stderr or "ubsan" in r.stderr:
            pytest.skip("no sanitizer runtimes: " + r.stderr.strip().splitlines()[-1])
        raise AssertionError(r.stderr)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1",
               LD_LIBRARY_PATH=os.path.join(CUDA, "lib64") + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr, run.stderr
    plans, images = (int(v) for v in run.stdout.split()[1::2])
    assert plans > 2000 and images > 900, run.stdout
