"""The C ABI library loads, exports every function include/fram.h declares,
and the Python structs match the C layouts (checked with gcc).  No GPU work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2508_00887_gb300 as fr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fram.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2508_00887_gb300 import build
    build.build()
    return fr.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fram_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ("fram_create", "fram_destroy", "fram_solve", "fram_solve_batched",
                     "fram_submit", "fram_poll", "fram_last_error", "fram_default_params"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", fr.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (fram_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert sorted(fr.exported_symbols()) == declared_functions()
    for n in declared_functions():
        assert hasattr(lib, n)


def _c_layout(struct, fields):
    body = "\n".join(f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    prog = f"""#include <stdio.h>
#include <stddef.h>
#include "fram.h"
int main(void) {{
  printf("%zu\\n", sizeof({struct}));
{body}
  return 0;
}}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("cname,pystruct,cfields", [
    ("fram_params", fr.FramParams,
     ["lambda", "alpha", "theta", "delta_tol", "gamma_tol", "polish_tol", "mixed_delta_tol",
      "stall_ratio", "stall_below", "max_outer",
      "max_sweeps", "max_polish", "precision", "init", "projection"]),
    ("fram_info", fr.FramInfo,
     ["outer_iters", "total_sweeps", "polish_sweeps", "sdsn_converged_last", "lap_augmentations",
      "lap_auction_phases", "delta", "gamma", "objective", "match_error", "assignment_value", "ms_total",
      "ms_gemm", "ms_sdsn", "ms_polish", "ms_update", "ms_rounding"]),
])
def test_struct_layouts_match_header(cname, pystruct, cfields):
    size, offs = _c_layout(cname, cfields)
    assert ctypes.sizeof(pystruct) == size
    pyoffs = [getattr(pystruct, name).offset for name, _ in pystruct._fields_]
    assert pyoffs == offs


def test_default_params_are_the_papers(lib):
    p = fr.fram_default_params()
    assert (p.lam, p.alpha, p.theta) == (1.0, 0.95, 10.0)     # Sec. 7 "Setting"
    assert p.delta_tol == 1e-6 and p.gamma_tol == 1e-14
    assert p.max_outer == 100 and p.max_sweeps == 200
    assert p.precision == fr.FRAM_PREC_FP64


def test_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    ctx = ctypes.c_void_p()
    st = lib.fram_create(ctypes.byref(ctx), 0, 0, None)
    assert st in (fr.FRAM_ERR_CUDA, fr.FRAM_ERR_INVALID)
    assert lib.fram_last_error(None) == b""


def test_binding_rejects_wrong_dtypes():
    import numpy as np
    with pytest.raises(ValueError):
        fr._addr(np.zeros((2, 2), dtype=np.float32))
    with pytest.raises(ValueError):
        fr._addr(np.zeros((4, 4))[:, :2])
    assert fr._addr(None) is None


def test_binding_takes_address_arrays_as_they_are():
    # fram_solve_batched's fast path: a numpy array of 8-byte addresses is
    # handed to the library without a copy; any other length is refused; a
    # list still goes through the per-entry checks.
    import numpy as np
    a = np.arange(5, dtype=np.uint64) * np.uint64(64) + np.uint64(4096)
    arg, keep = fr._ptr_table(a, 5, "float64")
    assert arg == a.ctypes.data and keep is a
    with pytest.raises(ValueError):
        fr._ptr_table(a, 4, "float64")
    arg, keep = fr._ptr_table([np.zeros((2, 2)), None], 2, "float64")
    assert len(arg) == 2 and arg[1] is None and arg is keep
    with pytest.raises(ValueError):
        fr._ptr_table([np.zeros((2, 2), dtype=np.float32)], 1, "float64")
    assert fr._ptr_table(None, 3, "float64") == (None, None)
    assert fr._is_index_array(np.zeros(3, dtype=np.int32), 4)
    assert not fr._is_index_array(np.zeros(3, dtype=np.float64), 8)
    assert not fr._is_index_array(np.zeros((2, 2), dtype=np.uint64), 8)
    assert not fr._is_index_array([1, 2, 3], 8)
