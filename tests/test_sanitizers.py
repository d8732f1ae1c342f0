"""Host code under AddressSanitizer and UBSan (CPU only; skipped where the compiler has no
sanitizer runtimes):

  * the planner (plan.cpp) and the job-image builder (program.cpp): tests/sanitize/
    planner_driver.cpp builds transform plans over a sweep of ring sizes, lengths, weights and
    both omega modes, and job images of every single-CTA and cluster shape;
  * the oracle (oracle/*.c): tests/sanitize/oracle_driver.c calls every entry point on small
    random inputs and checks the transforms against the DFT by definition and the products
    against schoolbook on the way (leak detection on).

An out-of-bounds access, a leak in the oracle or undefined behaviour fails the run."""
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


@pytest.mark.slow
def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("gcc is missing")
    exe = str(tmp_path / "oracle_driver")
    srcs = [os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c")] + [
        os.path.join(ROOT, "oracle", f) for f in ("ring.c", "transforms.c", "zx.c", "sn.c")]
    cmd = [cc, "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
           "-fno-omit-frame-pointer"] + srcs + ["-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "asan" in r.stderr or "ubsan" in r.stderr:
            pytest.skip("no sanitizer runtimes: " + r.stderr.strip().splitlines()[-1])
        raise AssertionError(r.stderr)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "runtime error" not in run.stderr and "Sanitizer" not in run.stderr, run.stderr
    counts = dict(zip(run.stdout.split()[0::2], (int(v) for v in run.stdout.split()[1::2])))
    assert counts["failures"] == 0 and counts["transforms"] > 100 and counts["products"] == 5, run.stdout
