"""The library used the way a CUDA C++ program uses it: its own kernels call the device
primitives (counting barrier, cohort mutex; and the GB300 defaults -- counting barrier, cluster
cohort mutex in both forms, ticket-window semaphore -- in cluster launches), the objects come
from the C ABI,
and the grids are launched through gsync_launch_coresident.  The program
(tests/cuda/user_kernel.cu) checks its own results exactly and prints OK."""
import os
import subprocess

import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_user_kernel_program(tmp_path):
    from paper_1110_4623_gb300 import build, gsync
    lib_dir = os.path.dirname(gsync.LIB_PATH)
    exe = tmp_path / "user_kernel"
    cmd = [build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
           "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "cuda", "user_kernel.cu"),
           "-L" + lib_dir, "-lgsync", "-Xlinker", "-rpath=" + lib_dir, "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
