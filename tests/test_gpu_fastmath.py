"""Device evaluation of the library's exp/log equals the host evaluation bit for bit,
on the table-driven range and on the inline out-of-range paths (the same code with
explicit fma and exact bit operations on both sides)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2508_16105_gb300 import build, rde_chem, synth

pytestmark = pytest.mark.gpu


def test_device_equals_host():
    build.build_library()
    lib = rde_chem.load_library()
    lib.rde_selftest_math.argtypes = [C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    for fn, x in ((0, synth.uniform_range(8, "e", 200000, -720.0, 720.0)),
                  (1, np.exp(synth.uniform_range(9, "l", 200000, -700.0, 700.0)))):
        host = np.empty_like(x)
        assert lib.rde_selftest_math(fn, x.size, x.ctypes.data, host.ctypes.data, 0, None) == 0
        dx = torch.as_tensor(x, device="cuda")
        dy = torch.empty_like(dx)
        s = torch.cuda.current_stream().cuda_stream
        assert lib.rde_selftest_math(fn, x.size, dx.data_ptr(), dy.data_ptr(), 1, s) == 0
        dev = dy.cpu().numpy()
        assert np.array_equal(dev.view(np.int64), host.view(np.int64))
