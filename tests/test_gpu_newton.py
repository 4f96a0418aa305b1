"""Float64 reciprocal square root and reciprocal by Newton-Raphson (the
helpers the top-k factorisations use in place of float64 division and square
root), on the GPU, against numpy's float64 1/sqrt(x) and 1/x (within one
rounding of the exact value) over the normal exponent range |e| <= 1022:
at most 4 units in the last place."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def newton(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("nr") / "libnewton_eval.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "gpu_fixture", "newton_eval.cu")], check=True)
    lib = ctypes.CDLL(out)
    lib.newton_eval.restype = ctypes.c_int
    lib.newton_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _ulps(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_newton_rsqrt_rcp_within_4_ulp(newton):
    rng = np.random.default_rng(5)
    n = 200_000
    mant = rng.uniform(1.0, 2.0, n)
    ex = rng.integers(-1021, 1022, n)
    x = np.ldexp(mant, ex)
    edge = np.array([1.0, 2.0, 4.0, 0.25, 3.0, 1e-300, 1e300, 2.0 ** -1021, 2.0 ** 1021,
                     np.nextafter(1.0, 2.0), np.nextafter(4.0, 0.0), 1.0 / 3.0])
    x = np.concatenate([x, edge, -x[:1000], -edge])
    xd = torch.as_tensor(x, device="cuda")
    rs = torch.empty_like(xd)
    rc = torch.empty_like(xd)
    assert newton.newton_eval(ctypes.c_void_p(xd.data_ptr()), x.size, ctypes.c_void_p(rs.data_ptr()),
                          ctypes.c_void_p(rc.data_ptr())) == 0
    rs, rc = rs.cpu().numpy(), rc.cpu().numpy()
    pos = x > 0
    assert _ulps(rs[pos], 1.0 / np.sqrt(x[pos])).max() <= 4.0
    assert _ulps(rc, 1.0 / x).max() <= 4.0
