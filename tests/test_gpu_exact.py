"""The preprocess evaluates the binning specification's two FP64 quantities - the scale
(float)exp((double)log_s) (step 5) and the alpha-footprint threshold
tau = (float)(2 ln(255 / (1 + exp(-logit)))) (step 14) - in float-float arithmetic with a
rounding-safety test and an FP64 fallback.  This compiles the library's header into a
small checker (tests/cuda/exact_check.cu) and requires the results to equal the FP64
expressions on 2^24 grid points and 2^24 scattered float bit patterns of [-60, 60]."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_float_float_matches_fp64_expressions(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "exact_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2509_17513_b300", "csrc"),
                    os.path.join(ROOT, "tests", "cuda", "exact_check.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe), str(1 << 24)], check=True, capture_output=True, text=True).stdout
    rows = [l.split() for l in out.splitlines() if l.startswith(("exp", "tau"))]
    assert len(rows) == 4, out
    for name, mode, n, mism, fall, err in rows:
        assert int(n) >= (1 << 23), (name, mode, n)
        assert int(mism) == 0, (name, mode, mism)
        assert int(fall) <= int(n) // 1000, (name, mode, fall)   # the FP64 fallback stays rare
        # float-float error well inside the margins of the safety test (2^-40 rel, 2^-37 abs)
        assert float(err) < (2.0 ** -42 if name == "exp" else 2.0 ** -40), (name, mode, err)
