"""The C ABI library loads without a GPU and exports every entry point of include/mh.h."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
from paper_2603_16721_gb300 import _build, mh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"MH_API\s+[\w\s\*]+?\b(mh_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_entry_points():
    names = _declared_symbols()
    for n in ("mh_create", "mh_create_device", "mh_solve", "mh_solve_ex", "mh_destroy", "mh_result_free",
              "mh_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_no_torch_types_in_header():
    for fn in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", fn)).read()
        assert "torch" not in text.replace("torch tensor", "").lower() or "at::" not in text
        assert "at::Tensor" not in text and "c10::" not in text


def test_argument_errors_need_no_gpu(lib):
    mh.load()
    with pytest.raises(mh.MHError) as e:
        mh.mh_solve(mh.Handle(None), 2)
    assert e.value.code == mh.MH_EINVAL
    assert "NULL" in mh.mh_last_error()
    bm = np.zeros((4, 2), dtype=np.uint64)
    with pytest.raises(mh.MHError) as e:
        mh.mh_create(bm, 4, 70000, 1)  # words do not match G*W
    assert e.value.code == mh.MH_EINVAL


def test_build_is_idempotent():
    t0 = os.path.getmtime(_build.LIB)
    __graft_entry__.build()
    assert os.path.getmtime(_build.LIB) == t0


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled against include/mh.h."""
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "mh.h"\n'
                   f'int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]


@pytest.mark.parametrize("struct,cls", [("mh_result", "mh_result"), ("mh_solve_opts", "mh_solve_opts"),
                                        ("mh_server_opts", "mh_server_opts"), ("mh_round_best", "mh_round_best")])
def test_binding_structs_match_header_layout(tmp_path, struct, cls):
    c = getattr(mh, cls)
    names = [f[0] for f in c._fields_]
    got = _c_layout(tmp_path, struct, names)
    assert got[0] == ctypes.sizeof(c)
    assert got[1:] == [getattr(c, n).offset for n in names]


def test_fault_specs_need_no_gpu(lib):
    mh.load()
    for ok in ("none", None, "alloc_fail=3", "timeout_after=1"):
        mh.mh_set_fault(ok)
    for bad in ("alloc_fail=0", "explode", "timeout_after=-2"):
        with pytest.raises(mh.MHError) as e:
            mh.mh_set_fault(bad)
        assert e.value.code == mh.MH_EINVAL and "alloc_fail" in str(e.value)
    mh.mh_set_fault(None)
