"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/hgks.h declares; without a GPU it fails loudly instead of falling
back to the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1909_01580_gb300 import build, hgks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgks_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hgks.EXPORTS)


def test_invalid_arguments_rejected_before_any_device_work():
    hgks.load()
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((0, 4, 4), (0, 0, 0), (1, 1, 1))
    assert e.value.code == hgks.HGKS_E_INVALID
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((4, 4, 4), (0, 0, 0), (1, 2, 1))  # non-cubic cells
    assert e.value.code == hgks.HGKS_E_INVALID
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((4, 4, 4), (0, 0, 0), (1, 1, 1), bc=(0, 1, 0, 0, 0, 0))  # unpaired periodic
    assert e.value.code == hgks.HGKS_E_INVALID
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((1025, 4, 4), (0, 0, 0), (1025, 4, 4))  # beyond HGKS_MAX_CELLS_PER_AXIS = 1024
    assert e.value.code == hgks.HGKS_E_INVALID
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((2, 8, 8), (0, 0, 0), (2, 8, 8), bc=(1, 1, 0, 0, 0, 0))  # reflective axis of 2 cells
    assert e.value.code == hgks.HGKS_E_INVALID


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_create((4, 4, 4), (0, 0, 0), (1, 1, 1))
    assert e.value.code == hgks.HGKS_E_CUDA
