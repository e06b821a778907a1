"""The geometry update divides by the small integer w + 1 with its correctly
rounded reciprocal and one residual correction instead of an IEEE division.
It must give the correctly rounded quotient for every weight and every
numerator the update can form; checked exhaustively on the device against
__fdiv_rn (see tests/gpu_checks/division_check.cu).  The geometry kernel
performs the same three operations on voxel pairs (__fmul2_rn, __ffma2_rn),
whose components round exactly as the scalar operations do, with the
reciprocal from rcp2_rn, which equals __frcp_rn (test_gpu_reciprocal.py)."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_division_by_weight_is_correctly_rounded(tmp_path):
    exe = str(tmp_path / "division_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false", "-std=c++17",
                           "-I", os.path.join(ROOT, "paper_1602_06645_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "gpu_checks", "division_check.cu"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 mismatches" in r.stdout
