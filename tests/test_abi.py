"""The C ABI library loads without a GPU and exports every entry point of include/mh.h."""
import ctypes
import os
import re

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
