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


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets the C compiler gives the
    header's structures."""
    import shutil
    import subprocess
    assert ctypes.sizeof(_binding.tg_hit) == 24
    structs = {"tg_hit": _binding.tg_hit, "tg_scan_opts": _binding.tg_scan_opts,
               "tg_outputs": _binding.tg_outputs}
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_version_and_status_strings(lib):
    assert "sm_103a" in tg.tg_version()
    assert tg.tg_abi_version() == 2
    assert tg.tg_status_string(tg.TG_ERR_TIMEOUT) == "device wait timed out"


def test_create_fails_loudly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tg.TgError):
        tg.tg_create(0)
