"""A look-back wait that nothing ends gives up: the bounded wait of the
single-pass stage-1 kernel (the allocation-free entry's).  A test build of that kernel
with a poll limit of 64 runs a document whose first tile no warp takes, so the
second tile waits on a status word that is never published; the wait must end
by itself, mark the document INTERNAL, and the kernel must finish (no fault,
no hang).  The build lives in a temporary directory."""
import ctypes
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_wait_with_nothing_to_end_it_gives_up():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1902_08318_gb300 as sj
    csrc = os.path.join(ROOT, "paper_1902_08318_gb300", "csrc")
    with tempfile.TemporaryDirectory() as tmp:
        so = os.path.join(tmp, "libbw.so")
        subprocess.check_call([sj._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-DSJ_SPIN_LIMIT=64",
                               "-I", os.path.join(ROOT, "include"), "-I", csrc,
                               os.path.join(ROOT, "tests", "bounded_wait.cu"),
                               os.path.join(csrc, "stage1.cu"), "-o", so])
        lib = ctypes.CDLL(so)
        lib.bw_run.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        flags = ctypes.c_uint32(0)
        assert lib.bw_run(ctypes.byref(flags)) == 0
        assert flags.value & 4  # kFlagInternal: the wait gave up
