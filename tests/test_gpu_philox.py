"""Pins the oracle's Philox4x32-10 to NVIDIA's cuRAND implementation (an
independent one): identical 128-bit outputs for random counters and keys,
including the counter layouts the annealer uses."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    from paper_2205_13399_gb300 import build
    out = os.path.join(tempfile.mkdtemp(), "philox_curand_probe.so")
    subprocess.run([build.nvcc()] + build.ARCH + ["-O2", "-Xcompiler", "-fPIC", "-shared",
                    os.path.join(HERE, "philox_curand_probe.cu"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    lib.philox_curand.restype = ctypes.c_int
    return lib


def test_oracle_philox_matches_curand(curand_lib):
    rng = np.random.default_rng(5)
    N = 2000
    ctr = rng.integers(0, 2 ** 32, size=(N, 4), dtype=np.uint64).astype(np.uint32)
    # cuRAND reaches counter word 1 through a 64-bit skip of 4 * (c0 + 2^32 c1)
    # outputs, so c1 stays below 2^30 here
    ctr[:, 1] >>= 2
    # the annealer's own counter shapes: (group, step, replica, tag)
    ctr[:500, 0] = rng.integers(0, 2048, 500)
    ctr[:500, 1] = rng.integers(0, 10 ** 6, 500)
    ctr[:500, 2] = rng.integers(0, 512, 500)
    ctr[:500, 3] = rng.integers(0, 5, 500)
    seeds = rng.integers(0, 2 ** 63, size=N, dtype=np.uint64)
    seeds[:10] = np.arange(10)
    out = np.zeros((N, 4), dtype=np.uint32)
    ctr = np.ascontiguousarray(ctr)
    rc = curand_lib.philox_curand(ctr.ctypes.data_as(ctypes.c_void_p),
                                  seeds.ctypes.data_as(ctypes.c_void_p),
                                  out.ctypes.data_as(ctypes.c_void_p), N)
    assert rc == 0
    for i in range(N):
        s = int(seeds[i])
        ref = oracle.philox(ctr[i], [s & 0xFFFFFFFF, s >> 32])
        assert np.array_equal(ref, out[i]), (i, ctr[i], s)
