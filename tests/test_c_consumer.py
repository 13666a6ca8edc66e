"""The boundary is a C ABI: a plain C99 program (tests/c/consumer.c) that
includes only include/tenergy.h compiles with gcc, links against the
in-tree libtenergy.so and runs (reporting TE_ECUDA where there is no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c99_consumer_builds_links_and_runs(tmp_path):
    from paper_2412_18553_gb300.build import build
    build()
    lib_dir = os.path.join(ROOT, "paper_2412_18553_gb300")
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    exe = str(tmp_path / "consumer")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "consumer.c"),
                    "-L", lib_dir, "-ltenergy", f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath-link,{cuda_lib}",
                    "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("create ")
