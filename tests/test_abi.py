"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/moda.h declares, and rejects bad arguments before
touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    import glob
    src = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(moda_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_13399_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    from paper_2205_13399_gb300 import moda
    assert _declared_functions() == sorted(moda.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_library_built_for_sm103a():
    from paper_2205_13399_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def _inst_args(n, F1=None, F2=None, D=None):
    rng = np.random.default_rng(n)
    if F1 is None:
        F1 = rng.integers(0, 100, (n, n)).astype(np.int16)
    if F2 is None:
        F2 = rng.integers(0, 100, (n, n)).astype(np.int16)
    if D is None:
        D = rng.integers(1, 100, (n, n))
        D = np.triu(D, 1)
        D = (D + D.T).astype(np.int16)
    return F1, F2, D


def _create(n, F1, F2, D, pen=None):
    from paper_2205_13399_gb300 import moda
    return moda.Instance(F1, F2, D, w=pen)


@pytest.mark.parametrize("case", ["n_small", "n_large", "negative", "asym", "diag", "kind"])
def test_create_instance_rejects_bad_input(case):
    from paper_2205_13399_gb300 import moda
    n = 6
    F1, F2, D = _inst_args(n)
    pen = None
    if case == "n_small":
        F1, F2, D = _inst_args(1)
    elif case == "n_large":
        F1, F2, D = _inst_args(129)
    elif case == "negative":
        F1 = F1.copy()
        F1[1, 2] = -1
    elif case == "asym":
        D = D.copy()
        D[0, 1] += 1
    elif case == "diag":
        D = D.copy()
        D[2, 2] = 5
    elif case == "kind":
        pen = (-1, 3)
    with pytest.raises(moda.MODAError) as ei:
        _create(n, F1, F2, D, pen)
    assert ei.value.status == moda.EINVAL


def test_create_instance_overflow():
    from paper_2205_13399_gb300 import moda
    n = 40
    F1 = np.full((n, n), 30000, dtype=np.int16)
    np.fill_diagonal(F1, 0)
    D = np.full((n, n), 30000, dtype=np.int16)
    np.fill_diagonal(D, 0)
    with pytest.raises(moda.MODAError) as ei:
        _create(n, F1, F1, D)
    assert ei.value.status == moda.EOVERFLOW


def test_null_arguments(lib):
    lib.moda_create_instance.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.moda_create_instance(4, None, None, None, None, ctypes.byref(out)) == 1
    lib.moda_anneal.restype = ctypes.c_int
    assert lib.moda_anneal(None, None, None, ctypes.byref(out)) == 1
    lib.moda_wait.restype = ctypes.c_int
    assert lib.moda_wait(None, ctypes.c_int64(0)) == 1
    lib.moda_last_error.restype = ctypes.c_char_p
    assert lib.moda_last_error()


def test_batch_and_server_null_arguments(lib):
    """Argument checks of the batch and serving entry points need no GPU."""
    P = ctypes.c_void_p
    out = ctypes.c_void_p()
    lib.moda_anneal_batch.restype = ctypes.c_int
    assert lib.moda_anneal_batch(None, None, 0, None, None) == 1
    lib.moda_server_create.restype = ctypes.c_int
    lib.moda_server_create.argtypes = [ctypes.c_size_t, P, P]
    assert lib.moda_server_create(0, None, None) == 1
    lib.moda_server_submit.restype = ctypes.c_int
    t = ctypes.c_int64()
    assert lib.moda_server_submit(None, None, None, ctypes.byref(t)) == 1
    lib.moda_server_poll.restype = ctypes.c_int
    lib.moda_server_poll.argtypes = [P, ctypes.c_int64, P]
    assert lib.moda_server_poll(None, 1, ctypes.byref(out)) == 1
    lib.moda_server_info.restype = ctypes.c_int
    assert lib.moda_server_info(None, None, None, None, None) == 1
    lib.moda_server_destroy.restype = None
    lib.moda_server_destroy(None)


def test_qubo_null_arguments(lib):
    P = ctypes.c_void_p
    out = ctypes.c_void_p()
    lib.moda_qubo_create.restype = ctypes.c_int
    assert lib.moda_qubo_create(2, 10, None, ctypes.byref(out)) == 1
    lib.moda_qubo_anneal.restype = ctypes.c_int
    assert lib.moda_qubo_anneal(None, None, None, ctypes.byref(out)) == 1
    lib.moda_qrun_wait.restype = ctypes.c_int
    assert lib.moda_qrun_wait(None) == 1
    lib.moda_qrun_read.restype = ctypes.c_int
    assert lib.moda_qrun_read(None, None, None, None, None, None, None, None) == 1
    lib.moda_qubo_destroy.restype = None
    lib.moda_qubo_destroy(None)
    lib.moda_qrun_destroy.restype = None
    lib.moda_qrun_destroy(None)


def test_kernel_variant_choice(tmp_path):
    """The host picks the kernel variants with the default algorithm or the
    placement compiled in only for runs that match them (a host-only C++
    check of moda::kernel_mode against the library's internal header)."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(os.path.dirname(here), "paper_2205_13399_gb300", "csrc")
    exe = str(tmp_path / "kernel_mode_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", cuda_inc,
                    os.path.join(here, "kernel_mode_check.cc"), "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout


def test_warp_layouts(tmp_path):
    """The warp engine's jump-record and shared-memory layouts, for every n
    and every buffer count the planner can choose: each part a bulk copy
    moves starts on a 16-byte boundary with a multiple of 16 bytes, the
    frozen-schedule layout stays inside the buffer region, and no parts
    overlap (a host-only C++ check against the library's internal
    header)."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(os.path.dirname(here), "paper_2205_13399_gb300", "csrc")
    exe = str(tmp_path / "warp_layout_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", cuda_inc,
                    os.path.join(here, "warp_layout_check.cc"), "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout


def test_check_accept_rejects_bad_arguments():
    """moda_check_accept validates every input before any device work."""
    from paper_2205_13399_gb300 import moda
    for a, d, i in (([-1], [1.0], [0]), ([1], [0.0], [0]), ([1], [1.0], [65536]),
                    ([1], [float("inf")], [3])):
        with pytest.raises(moda.MODAError) as ei:
            moda.check_accept(a, d, i)
        assert ei.value.status == moda.EINVAL
