"""The FP64 reciprocal of the round kernels (devutil.cuh: a float seed and one step of Chebyshev's
third-order iteration y (1 + e + e^2), e = 1 - d y) against CUDA's IEEE double division, on the GPU:
within one unit in the last place for operands over the exponent range the fast path covers, both
signs, mantissas at and near the binade ends, and the fallback range."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include "devutil.cuh"
__global__ void k_rcp(int n, const double *d, double *y, double *ref) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { y[i] = gabp::rcp64(d[i]); ref[i] = 1.0 / d[i]; }
}
extern "C" int rcp_check(int n, const double *d, double *y, double *ref) {
  k_rcp<<<(n + 255) / 256, 256>>>(n, d, y, ref);
  return (int)cudaDeviceSynchronize();
}
'''


@pytest.fixture(scope="module")
def rcp_lib():
    tmp = tempfile.mkdtemp()
    cu, so = os.path.join(tmp, "rcp.cu"), os.path.join(tmp, "rcp.so")
    open(cu, "w").write(SRC)
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                    "-I", os.path.join(ROOT, "paper_0811_2518_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-o", so, cu], check=True)
    lib = ctypes.CDLL(so)
    lib.rcp_check.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.rcp_check.restype = ctypes.c_int
    return lib


def test_rcp64_within_one_ulp(rcp_lib):
    rng = np.random.default_rng(3)
    m = rng.uniform(1.0, 2.0, 1_000_000)
    e = rng.integers(-125, 126, m.size)
    d = np.ldexp(m, e) * rng.choice([-1.0, 1.0], m.size)
    ends = np.array([1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5, 1.0 + 2.0 ** -20, 1.0 + 2.0 ** -21,
                     2.0 - 2.0 ** -20, 3.0, 7.0, 0.1, 1e-30, 1e30, 2.0 ** 120, 2.0 ** -120, 2.0 ** 121, 2.0 ** -121,
                     1e-300, 1e300])
    d = np.concatenate([d, ends, -ends])
    dt = torch.from_numpy(d).cuda()
    y = torch.empty_like(dt)
    ref = torch.empty_like(dt)
    assert rcp_lib.rcp_check(d.size, dt.data_ptr(), y.data_ptr(), ref.data_ptr()) == 0
    y, ref = y.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(y))
    assert np.all(np.abs(y - ref) <= np.spacing(np.abs(ref)))
