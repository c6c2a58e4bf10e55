"""The C ABI without a GPU: the library builds, loads and exports every entry point that
include/sprot.h declares, and the ctypes structures match the C layouts (not gpu)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2502_06337_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sprot.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sprot_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sprot_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    lib = binding.load(libpath)
    for name in binding.EXPORTS:
        assert hasattr(lib, name)
    assert binding.status_text(binding.E_NOAXIS).startswith("no axis")
    p = binding.Params()
    lib.sprot_default_params(ctypes.byref(p))
    assert (p.grid, p.angle_bins, p.k, p.gate_window, p.angle_window) == (256, 360, 1, 1, 1)
    assert lib.sprot_autotune_grid(1000) == 128 and lib.sprot_autotune_grid(10**6) == 512


def test_struct_layouts_match_c(libpath, tmp_path):
    """sizeof/offsetof of every ABI struct, compiled from the header with gcc."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sprot.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(sprot_params), sizeof(sprot_rotation), sizeof(sprot_debug), sizeof(sprot_instance),"
        "sizeof(sprot_server_cfg), sizeof(sprot_request), sizeof(sprot_result),"
        "offsetof(sprot_params, tau), offsetof(sprot_rotation, cell_row), offsetof(sprot_result, t_submit_ms));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(binding.Params), ctypes.sizeof(binding.Rotation), ctypes.sizeof(binding.Debug),
            ctypes.sizeof(binding.Instance), ctypes.sizeof(binding.ServerCfg),
            ctypes.sizeof(binding.Request), ctypes.sizeof(binding.Result),
            binding.Params.tau.offset, binding.Rotation.cell_row.offset, binding.Result.t_submit_ms.offset]
    assert got == want


def test_invalid_arguments_rejected_without_gpu(libpath):
    """Argument checks run before any CUDA call."""
    lib = binding.load(libpath)
    p = binding.make_params(grid=100)  # not a power of two
    out = binding.Rotation()
    assert lib.sprot_estimate_rotation(None, None, 10, ctypes.byref(p), ctypes.byref(out), None, None) == binding.E_INVAL
    assert lib.sprot_axis_vote(None, None, 0, 256, None, None) == binding.E_INVAL
