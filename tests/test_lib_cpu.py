"""CPU checks of the C-ABI library: it loads, exports every function that
include/hhignn.h declares, and fails cleanly (no crash) without a GPU."""
import ctypes
import os
import re

import pytest

import paper_2505_08174_b300 as hh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hhignn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(hh.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = hh.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_default_params_host_only():
    p = hh.Params()
    assert (p.leaf_size, p.eta, p.eps, p.max_rank, p.n_shards) == (32, 1.0, 1e-4, 48, 1)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    st = hh.lib().hh_create(ctypes.byref(h), 0)
    assert st in (hh.HH_ERR_CUDA, hh.HH_ERR_ARG) and not h.value
