"""The C-ABI library: builds, loads, exports every declared symbol, and
rejects bad input on the host before touching a GPU (no compute calls)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1701_06588_gb300 import _lib as L
from paper_1701_06588_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "shg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 15
    bound = {n for n, _, _ in L.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n
        assert n in bound, "no Python binding for " + n
    assert L.shg_version().startswith("shg-gb300")


def _shells(**kw):
    d = dict(l=np.array([0, 1], np.int32), nprim=np.array([1, 2], np.int32), exps=np.array([1.0, 2.0, 0.5]),
             coefs=np.array([1.0, 0.3, -0.2]), centers=np.zeros((2, 3)), center_of=np.array([0, 1], np.int32))
    d.update(kw)
    return d


@pytest.mark.parametrize("bad,msg", [
    (dict(l=np.array([0, 7], np.int32)), "l = 7"),
    (dict(l=np.array([-1, 1], np.int32)), "l = -1"),
    (dict(nprim=np.array([0, 3], np.int32), exps=np.array([1.0, 2.0, 0.5]), coefs=np.ones(3)), "K = 0"),
    (dict(nprim=np.array([33, 1], np.int32), exps=np.ones(34), coefs=np.ones(34)), "K = 33"),
    (dict(exps=np.array([1.0, -2.0, 0.5])), "exponent"),
    (dict(exps=np.array([1.0, math.nan, 0.5])), "exponent"),
    (dict(coefs=np.array([1.0, math.inf, 0.5])), "coefficient"),
    (dict(centers=np.array([[0, 0, 0], [0, math.nan, 0]], float)), "center coordinate"),
    (dict(center_of=np.array([0, 2], np.int32)), "center index"),
])
def test_basis_validation_on_host(lib, bad, msg):
    s = _shells(**bad)
    with pytest.raises(L.ShgError) as e:
        L.shg_basis_create(len(s["l"]), s["l"], s["nprim"], s["exps"], s["coefs"], len(s["centers"]),
                           np.ascontiguousarray(s["centers"], dtype=np.float64), s["center_of"], 1)
    assert e.value.code == L.SHG_EINVAL
    assert msg in str(e.value)


def test_null_and_range_arguments(lib):
    assert lib.shg_basis_create(0, None, None, None, None, 0, None, None, 1, ctypes.byref(ctypes.c_void_p())) == L.SHG_EINVAL
    assert lib.shg_basis_create(1, None, None, None, None, 1, None, None, 1, None) == L.SHG_EINVAL
    assert lib.shg_plan_2c_create(None, 10, None, None, 1, None, ctypes.byref(ctypes.c_void_p())) == L.SHG_EINVAL
    assert lib.shg_plan_2c_exec(None, 0, 0.0, 0.0, 0, None, None, None) == L.SHG_EINVAL
    assert lib.shg_pair_offsets(None, 1, None, None, None) == L.SHG_EINVAL
    ops = (ctypes.c_int * 2)(1, 2)
    om = (ctypes.c_double * 2)(0.0, 0.1)
    assert lib.shg_plan_2c_exec_fused(None, 2, ops, om, 0, None, None, None) == L.SHG_EINVAL
    assert "plan is NULL" in L.shg_last_error()
    assert lib.shg_graph_2c_create_fused(None, 2, ops, om, 1, None, None, ctypes.byref(ctypes.c_void_p())) == L.SHG_EINVAL
    assert lib.shg_graph_2c_create_fused(None, 2, ops, om, 0, None, None, None) == L.SHG_EINVAL
    assert lib.shg_debug_boys(10, None, 99, None, None) == L.SHG_EINVAL
    assert "nmax" in L.shg_last_error()
    lib.shg_basis_destroy(None)
    lib.shg_plan_destroy(None)
    assert lib.shg_basis_nshells(None) == 0
