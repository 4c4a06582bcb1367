"""The C ABI library builds for sm_103a, loads, and exports every entry point of include/tg.h.

No computation is launched here (this runs without a GPU).
"""
import ctypes
import os
import re
import shutil

import pytest

import paper_2604_21095_gb300 as tg
from paper_2604_21095_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tg.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit to build the library")
    tg.build()
    return tg.load()


def test_header_declares_the_scan_calls():
    names = _declared()
    for required in ("tg_prepare_panel", "tg_scan_block", "tg_decode_block", "tg_scan_host",
                     "tg_create", "tg_destroy", "tg_status_poll", "tg_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_the_header():
    assert sorted(_binding.exported_symbols()) == _declared()


def test_struct_layouts_match_header():
    assert ctypes.sizeof(_binding.tg_hit) == 24
    assert ctypes.sizeof(_binding.tg_scan_opts) == 16
    assert ctypes.sizeof(_binding.tg_outputs) == 12 * 8


def test_version_and_status_strings(lib):
    assert "sm_103a" in tg.tg_version()
    assert tg.tg_abi_version() == 1
    assert tg.tg_status_string(tg.TG_ERR_TIMEOUT) == "device wait timed out"


def test_create_fails_loudly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tg.TgError):
        tg.tg_create(0)
