"""The C client (tests/c/onmf_c_smoke.c) built with gcc against
include/onmf.h and linked to libonmf.so: an online pass over host frames in
FP32 and mixed precision and a projection through the plain C ABI."""
import os
import shutil
import subprocess

import pytest

import paper_1106_4198_gb300 as onmf

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_runs(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    lib = onmf._build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "onmf_c_smoke")
    subprocess.run(["gcc", "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "onmf_c_smoke.c"), "-o", exe,
                    "-L", libdir, "-l:" + os.path.basename(lib), "-lm",
                    "-Wl,-rpath," + libdir], check=True)
    env = dict(os.environ)
    cuda_lib = "/usr/local/cuda/lib64"
    env["LD_LIBRARY_PATH"] = ":".join(p for p in (libdir, cuda_lib, env.get("LD_LIBRARY_PATH"))
                                      if p)
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
