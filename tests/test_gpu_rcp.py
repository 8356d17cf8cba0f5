"""The ratio bounds of the bound pass take reciprocals with the hardware approximation
rcp.approx.ftz.f32 and widen their results by its error bound (2^-23 relative).  This test
checks that bound exhaustively over every normal input the kernel can pass, [2^-126, 2^120]."""
import ctypes as C
import os
import struct
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def test_rcp_approx_relative_error_is_at_most_one_ulp(tmp_path):
    so = tmp_path / "rcp_probe.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                    "-o", str(so), os.path.join(HERE, "rcp_probe.cu")], check=True)
    L = C.CDLL(str(so))
    L.rcp_max_rel_err.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_double)]
    out = C.c_double()
    lo, hi = bits(2.0 ** -126), bits(2.0 ** 120)
    assert L.rcp_max_rel_err(lo, hi, C.byref(out)) == 0
    print("max relative error of rcp.approx.ftz.f32 on [2^-126, 2^120]:", out.value, "=", out.value / 2.0 ** -23,
          "x 2^-23")
    assert 0.0 < out.value <= 2.0 ** -23
