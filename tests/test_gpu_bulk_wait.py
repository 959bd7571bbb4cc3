"""The bounded wait of the bulk shared-memory copies (csrc/bulk_copy.cuh), through a test-only probe
kernel built here from tests/bulk_wait_probe.cu: a real copy completes and arrives intact with status
0; a barrier that expects bytes no copy delivers makes the wait give up within its poll limit, which
sets status bit 1 without a fault, and the context stays usable afterwards."""
import ctypes
import os
import subprocess
import tempfile
import time

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe():
    out = os.path.join(tempfile.mkdtemp(prefix="bulkprobe_"), "libbulkprobe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "bulk_wait_probe.cu")], check=True)
    lib = ctypes.CDLL(out)
    lib.probe_bulk_copy.restype = ctypes.c_int
    lib.probe_bulk_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]
    return lib


def _run(lib, n, extra):
    src = torch.arange(n, dtype=torch.float32, device="cuda") * 0.5 + 1.0
    dst = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    code = lib.probe_bulk_copy(src.data_ptr(), dst.data_ptr(), n, extra, status.data_ptr())
    return code, time.perf_counter() - t0, src, dst, int(status.item())


def test_bulk_copy_completes(probe):
    code, _, src, dst, status = _run(probe, 5120, 0)      # one p = 7 element's state, 20 KB
    assert code == 0 and status == 0
    assert torch.equal(src, dst)


def test_bounded_wait_gives_up_and_reports(probe):
    code, seconds, _, dst, status = _run(probe, 1024, 16)
    assert code == 0, "the probe must return without a fault"
    assert status == 1
    assert bool((dst == -7.0).all()), "the element is left unevaluated"
    assert seconds < 30.0
    # the context is still usable
    x = torch.ones(1 << 20, device="cuda")
    assert float(x.sum()) == float(1 << 20)
    code, _, src, dst, status = _run(probe, 256, 0)
    assert code == 0 and status == 0 and torch.equal(src, dst)
