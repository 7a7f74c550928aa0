"""Host-side checks of the chemistry kernel's numerical helpers: the integer
float<->double conversions (against the conversion instructions, every
float; ties and carries for doubles) and the rate table evaluated the
kernel's way against the rate fits in long double.  Compiled with nvcc,
run on the CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_host_numerics(tmp_path):
    exe = tmp_path / "host_numerics"
    src = os.path.join(ROOT, "tests", "host_numerics.cu")
    tab = os.path.join(ROOT, "paper_1508_07888_b300", "csrc", "rate_table.cu")
    subprocess.run(["nvcc", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", str(exe), src, tab], check=True, capture_output=True, timeout=600)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "OK" in r.stdout
