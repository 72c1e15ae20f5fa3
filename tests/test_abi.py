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


STRUCTS = [("ricmrcc_layout", "Layout"), ("ricmrcc_opts", "Opts"), ("ricmrcc_stats", "Stats"),
           ("ricmrcc_plan_info_t", "PlanInfo"), ("ricmrcc_tile_rule", "TileRule"), ("ricmrcc_tuning", "Tuning"),
           ("ricmrcc_batch_info_t", "BatchInfo"), ("ricmrcc_ladder_info_t", "LadderInfo"),
           ("ricmrcc_adjoint_info", "AdjointInfo")]


def test_binding_structs_match_the_header(tmp_path):
    """sizeof of every ABI struct (C compiler, the header as shipped) equals
    the ctypes layout the binding passes."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    inc = os.path.join(os.path.dirname(here), "include")
    src = tmp_path / "sizes.c"
    body = "".join(f'  printf("{c} %zu\\n", sizeof({c}));\n' for c, _ in STRUCTS)
    src.write_text("#include <stdio.h>\n#include \"ricmrcc.h\"\nint main(void) {\n" + body + "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = dict(zip(out[0::2], (int(x) for x in out[1::2])))
    for c, py in STRUCTS:
        assert sizes[c] == ctypes.sizeof(getattr(ric, py)), (c, sizes[c], ctypes.sizeof(getattr(ric, py)))


def test_emulated_gemm_and_adjoint_info_argument_errors(lib_path):
    """Refused before any device work."""
    lib = ric.load_library()
    f = lib.ricmrcc_gemm_f64_emulated
    assert f(None, 1, None, 1, None, 1, -1, 1, 1, 1.0, 0, None) == ric.EINVAL
    assert f(None, 1, None, 1, None, 1, 1, 1, 1, 1.0, ric_max_slices() + 1, None) == ric.EINVAL
    assert f(None, 1, None, 1, None, 1, 1, 1, 1, float("nan"), 0, None) == ric.EINVAL
    assert f(None, 1, None, 1, None, 1, 4, 4, 4, 1.0, 0, None) == ric.EINVAL  # null operands
    assert f(None, 1, None, 1, None, 1, 0, 4, 4, 1.0, 0, None) == ric.OK     # empty: nothing to do
    assert lib.ricmrcc_get_adjoint_info(None, None) == ric.EINVAL


def ric_max_slices():
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(os.path.dirname(here), "include", "ricmrcc.h")).read()
    return int(re.search(r"#define RICMRCC_EMULATED_MAX_SLICES (\d+)", text).group(1))
