"""The geometry update projects voxels with its own correctly rounded
reciprocal (the hardware's approximate reciprocal and one Newton step, on
voxel pairs) instead of __frcp_rn.  It must equal __frcp_rn for every binary32
in [2^-126, 2^126), every value whose reciprocal is a normal number; checked
exhaustively on the device (see tests/gpu_checks/reciprocal_check.cu).
Voxel depths lie far inside that range (the library keeps volumes and camera
translations within 10^6 m); a depth of zero or below fails the projection's
Z > 0 test before the reciprocal matters."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reciprocal_is_correctly_rounded(tmp_path):
    exe = str(tmp_path / "reciprocal_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "--fmad=false", "-std=c++17",
                           "-I", os.path.join(ROOT, "paper_1602_06645_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "gpu_checks", "reciprocal_check.cu"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 mismatches" in r.stdout
