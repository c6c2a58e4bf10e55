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
        "printf(\"%zu %zu\\n\", sizeof(sprot_plan_knobs), offsetof(sprot_plan_knobs, ms_tuned));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(binding.Params), ctypes.sizeof(binding.Rotation), ctypes.sizeof(binding.Debug),
            ctypes.sizeof(binding.Instance), ctypes.sizeof(binding.ServerCfg),
            ctypes.sizeof(binding.Request), ctypes.sizeof(binding.Result),
            binding.Params.tau.offset, binding.Rotation.cell_row.offset, binding.Result.t_submit_ms.offset,
            ctypes.sizeof(binding.Knobs), binding.Knobs.ms_tuned.offset]
    assert got == want


def test_plan_knobs_without_gpu(libpath):
    """The default knobs, and the tuned-plan query without a device (nothing tuned: the
    defaults); the tuners check their arguments before any CUDA call."""
    lib = binding.load(libpath)
    assert binding.default_knobs() == {"vote_rounds": 1, "chunk_div": 600, "batch_slice": 32768,
                                       "batch_div": 1200, "ms_tuned": 0.0, "ms_default": 0.0}
    binding.autotune_reset()
    found, k = binding.tuned_plan(10**6, 512)
    assert not found and k == binding.default_knobs()
    p = binding.make_params()
    kn = binding.Knobs()
    for reps in (0, 16):
        assert lib.sprot_autotune_plan(FAKE, FAKE, 1000, ctypes.byref(p), reps, ctypes.byref(kn), None) == binding.E_INVAL
    assert lib.sprot_autotune_plan(FAKE, FAKE, 0, ctypes.byref(p), 3, ctypes.byref(kn), None) == binding.E_INVAL
    assert lib.sprot_autotune_batch(None, 4, 3, ctypes.byref(kn), None) == binding.E_INVAL
    for field, value in (("vote_rounds", 0), ("vote_rounds", 4), ("chunk_div", 99), ("chunk_div", 2401),
                         ("batch_slice", 16383), ("batch_slice", 65536), ("batch_div", 299), ("batch_div", 4801)):
        bad = binding.Knobs(1, 600, 32768, 1200, 0.0, 0.0)
        setattr(bad, field, value)
        assert lib.sprot_set_tuned_plan(1000, 256, 0, ctypes.byref(bad)) == binding.E_INVAL
    good = binding.Knobs(1, 600, 32768, 1200, 0.0, 0.0)
    assert lib.sprot_set_tuned_plan(1000, 100, 0, ctypes.byref(good)) == binding.E_INVAL  # G not a power of two


def test_invalid_arguments_rejected_without_gpu(libpath):
    """Argument checks run before any CUDA call."""
    lib = binding.load(libpath)
    p = binding.make_params(grid=100)  # not a power of two
    out = binding.Rotation()
    assert lib.sprot_estimate_rotation(None, None, 10, ctypes.byref(p), ctypes.byref(out), None, None) == binding.E_INVAL
    assert lib.sprot_axis_vote(None, None, 0, 256, None, None) == binding.E_INVAL


# A stand-in input pointer that is never dereferenced: every call below must fail its host-side
# argument checks (E_INVAL) before any CUDA call; a case that passed them would reach CUDA with it.
FAKE = ctypes.c_void_p(0x1000)


@pytest.mark.parametrize("field,value", [
    ("grid", 24), ("grid", 8), ("grid", 4096), ("grid", -256),
    ("angle_bins", 1), ("angle_bins", 5000),
    ("k", 0), ("k", 9),
    ("tau", 0.0), ("tau", -1.0), ("tau", float("nan")), ("tau", float("inf")),
    ("nms_deg", -1.0), ("nms_deg", float("nan")),
    ("gate_window", -2), ("angle_window", -1),
    ("flags", 0x80),
])
def test_every_parameter_is_checked_before_any_cuda_call(libpath, field, value):
    lib = binding.load(libpath)
    p = binding.make_params(grid=256, angle_bins=360, k=1, nms_deg=2.0, tau=0.05)
    setattr(p, field, value)
    outs = (binding.Rotation * 9)()
    nf = ctypes.c_int32(0)
    assert lib.sprot_estimate_rotations_ex(FAKE, FAKE, 1000, ctypes.byref(p), outs, ctypes.byref(nf), None, None,
                                           None) == binding.E_INVAL
    if field != "k":  # the single-rotation entry forces k = 1
        assert lib.sprot_estimate_rotation(FAKE, FAKE, 1000, ctypes.byref(p), outs, None, None) == binding.E_INVAL


@pytest.mark.parametrize("n", [0, -5, (1 << 31) + 1])
def test_pair_counts_are_checked(libpath, n):
    lib = binding.load(libpath)
    p = binding.make_params()
    out = binding.Rotation()
    assert lib.sprot_estimate_rotation(FAKE, FAKE, n, ctypes.byref(p), ctypes.byref(out), None, None) == binding.E_INVAL


def test_structural_argument_checks(libpath):
    lib = binding.load(libpath)
    p = binding.make_params()
    out = binding.Rotation()
    nf = ctypes.c_int32(0)
    E = binding.E_INVAL
    assert lib.sprot_estimate_rotation(FAKE, FAKE, 10, None, ctypes.byref(out), None, None) == E
    assert lib.sprot_estimate_rotation(FAKE, FAKE, 10, ctypes.byref(p), None, None, None) == E
    assert lib.sprot_estimate_rotation(None, FAKE, 10, ctypes.byref(p), ctypes.byref(out), None, None) == E
    assert lib.sprot_estimate_rotation(FAKE, None, 10, ctypes.byref(p), ctypes.byref(out), None, None) == E
    # host inputs cannot export device debug buffers
    ph = binding.make_params(flags=binding.HOST_PTRS)
    dbg = binding.Debug(None, None, None, None)
    assert lib.sprot_estimate_rotations_ex(FAKE, FAKE, 10, ctypes.byref(ph), ctypes.byref(out), ctypes.byref(nf),
                                           None, ctypes.byref(dbg), None) == E
    # batches: empty, null, an instance with host pointers, an invalid instance after a valid one
    assert lib.sprot_estimate_batch(None, 1, None) == E
    inst = (binding.Instance * 2)()
    assert lib.sprot_estimate_batch(inst, 0, None) == E
    for i in range(2):
        inst[i].P, inst[i].Q, inst[i].n = FAKE.value, FAKE.value, 100
        inst[i].params = binding.make_params()
        inst[i].out = ctypes.pointer(out)
    inst[1].params.flags = binding.HOST_PTRS
    assert lib.sprot_estimate_batch(inst, 2, None) == E
    inst[1].params = binding.make_params(angle_bins=1)
    assert lib.sprot_estimate_batch(inst, 2, None) == E
    # stage entry points
    assert lib.sprot_axis_vote(FAKE, FAKE, 10, 100, FAKE, None) == E            # G not a power of two
    assert lib.sprot_axis_vote_sampled(FAKE, FAKE, 10, 64, 0, FAKE, None) == E  # J < 1
    assert lib.sprot_axis_vote_sampled(FAKE, FAKE, 10, 64, 5000, FAKE, None) == E
    assert lib.sprot_axis_vote_eps(FAKE, FAKE, 10, 64, -0.1, FAKE, None) == E  # eps < 0
    assert lib.sprot_select_peaks(FAKE, 64, 0, 2.0, FAKE, FAKE, FAKE, None) == E  # k < 1


def test_status_strings_and_defaults(libpath):
    lib = binding.load(libpath)
    codes = [binding.OK, binding.E_INVAL, binding.E_NOMEM, binding.E_CUDA, binding.E_TIMEOUT, binding.E_NOAXIS,
             binding.E_UNIMPL, binding.E_BUSY]
    texts = [lib.sprot_status_string(c).decode() for c in codes]
    assert len(set(texts)) == len(codes) and all(texts)
    p = binding.Params()
    lib.sprot_default_params(ctypes.byref(p))
    assert (p.grid, p.angle_bins, p.k, p.gate_window, p.angle_window, p.flags) == (256, 360, 1, 1, 1, 0)
    assert abs(p.nms_deg - 2.0) < 1e-6 and abs(p.tau - 0.05) < 1e-12
    assert [lib.sprot_autotune_grid(n) for n in (1, 2999, 3000, 299999, 300000, 10**7)] == [128, 128, 256, 256, 512, 512]
