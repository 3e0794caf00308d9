"""pdst_stream_read, the benchmark's streaming-read ceiling, through the C ABI:
it runs on a buffer larger than L2 and rejects sizes and addresses that its
16-byte loads cannot take."""
import ctypes

import pytest

from paper_2604_11920_b300 import pdst
from gpu_util import require_cuda

pytestmark = pytest.mark.gpu


def test_stream_read_runs_and_checks_arguments():
    require_cuda()
    import torch
    buf = torch.rand(64 << 20, device="cuda", dtype=torch.float32)   # 256 MB
    pdst.stream_read(buf)
    torch.cuda.synchronize()
    lib = pdst.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.pdst_stream_read(ctypes.c_void_p(buf.data_ptr()), 100, stream) == 1
    assert lib.pdst_stream_read(ctypes.c_void_p(buf.data_ptr() + 4), 1024, stream) == 1
    assert lib.pdst_stream_read(None, 1024, stream) == 1
    assert lib.pdst_stream_read(ctypes.c_void_p(buf.data_ptr()), 0, stream) == 0
    torch.cuda.synchronize()
