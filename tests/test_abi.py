"""The C-ABI library builds, loads and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

import paper_2511_03567_gb300 as ric
from paper_2511_03567_gb300 import build as B


@pytest.fixture(scope="module")
def lib_path():
    try:
        return B.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc here
        pytest.skip(f"cannot build: {e}")


def test_library_exports_every_header_symbol(lib_path):
    declared = set(ric.header_symbols())
    assert len(declared) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared <= exported, declared - exported
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert getattr(lib, name) is not None


def test_binding_declares_every_symbol(lib_path):
    lib = ric.load_library()
    for name in ric.header_symbols():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert fn.restype is not None or name.endswith("_destroy"), name


def test_argument_errors_without_gpu(lib_path):
    lib = ric.load_library()
    h = ctypes.c_void_p()
    assert lib.ricmrcc_create(-1, 2, 3, 4, ctypes.byref(h)) == ric.EINVAL
    assert lib.ricmrcc_create(1, 2, 3, 0, ctypes.byref(h)) == ric.EINVAL
    # batch sizes are validated before any device work
    dims = (ctypes.c_int * 8)(2, 4, 10, 48, 1, 2, 3, 0)
    b = ctypes.c_void_p()
    assert lib.ricmrcc_batch_create(0, dims, ctypes.byref(b)) == ric.EINVAL
    assert lib.ricmrcc_batch_create(2, dims, ctypes.byref(b)) == ric.EINVAL  # n_aux = 0
    assert lib.ricmrcc_batch_create(1, None, ctypes.byref(b)) == ric.EINVAL
    assert lib.ricmrcc_batch_create(1, dims, None) == ric.EINVAL
    assert lib.ricmrcc_tune(None, 0, 1, None) == ric.EINVAL
    assert lib.ricmrcc_batch_residual(None, 0, None) == ric.EINVAL
    o = ric.Opts()
    assert lib.ricmrcc_opts_default(ctypes.byref(o)) == ric.OK
    assert o.s == 0.5 and o.max_iter == 100 and o.diis_size == 8
