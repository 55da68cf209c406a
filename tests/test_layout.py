"""Host-side properties of the tensor-core forms' layout (no GPU): the map from a point's form
index to its stored position keeps every block of 128 points in place and gives each MMA quad
lane a quarter of 32 consecutive points (what the candidate re-checks read), and the staging
threads' point order writes whole groups of forms. tests/host_layout_check.cu states them and
is compiled against the library's internal header."""
import os
import subprocess

import pytest

from paper_2204_03139_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_form_layout_maps(tmp_path):
    try:
        cc = build.nvcc()
    except RuntimeError as e:
        pytest.skip(str(e))
    exe = str(tmp_path / "host_layout_check")
    r = subprocess.run([cc, *build.ARCH, "-std=c++17", "-o", exe,
                        os.path.join(HERE, "host_layout_check.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
