"""Host-only checks of the C ABI: the library loads without a GPU and
exports every entry point that include/mcdesign.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mcdesign.h")


def declared():
    text = open(HEADER).read()
    return re.findall(r"^\s*(?:mcd_status|void|const char\*|int64_t)\s+(\w+)\(", text, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2005_10494_gb300 import build
    path = build.build()
    import paper_2005_10494_gb300 as pkg
    return pkg.load(path)


def test_header_declares_the_boundary():
    names = set(declared())
    for n in ["mc_design_eval", "mc_design_grad", "mc_smooth_argmax", "mcd_plan_create", "mcd_plan_eval",
              "mcd_plan_grad", "mcd_plan_destroy", "mcd_create", "mcd_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    assert set(declared()) <= exported
    # nothing else of the C ABI namespace leaks out
    assert {s for s in exported if s.startswith(("mc_", "mcd_"))} == set(declared())


def test_header_compiles_as_c():
    src = '#include "mcdesign.h"\nint main(void) { mcd_problem p; (void)p; return MCD_OK; }\n'
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), "-x", "c", "-",
                        "-o", "/dev/null"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_no_device_reports_an_error(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = lib.mcd_create(ctypes.byref(h), 0)
    assert rc != 0 and not h.value


def test_package_raises_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2005_10494_gb300 as pkg
    with pytest.raises(RuntimeError):
        pkg.Context(0)


def test_oracle_is_independent_of_the_cuda_path():
    # the oracle shares no code with the CUDA library and neither imports the other
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "paper_2005_10494_gb300" not in text and "csrc" not in text, f
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2005_10494_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("oracle's", ""), f


def test_binding_constants_match_the_header():
    import paper_2005_10494_gb300.binding as b
    text = open(HEADER).read()
    defs = dict(re.findall(r"^#define\s+(MCD_\w+)\s+(-?\d+)", text, re.M))
    for name, val in defs.items():
        if hasattr(b, name):
            assert getattr(b, name) == int(val), name
    for name in ["MCD_PLAN_GRAD", "MCD_PLAN_AUTOTUNE", "MCD_PLAN_GRAPH", "MCD_PLAN_FP64", "MCD_PLAN_TIMING",
                 "MCD_PLAN_SHARED", "MCD_SHARED_MIN", "MCD_MAX_D", "MCD_ANY_EXCEEDS", "MCD_ALL_BELOW"]:
        assert name in defs and hasattr(b, name), name


def test_pipe_classes_match_the_header():
    """binding.PIPE_CLASSES lists the MCD_PIPE_* classes in header order, and
    bench.py's per-draw counts use only measured classes."""
    import bench
    import paper_2005_10494_gb300.binding as b
    text = open(HEADER).read()
    defs = {k: int(v) for k, v in re.findall(r"^#define\s+MCD_PIPE_(\w+)\s+(\d+)", text, re.M)}
    count = defs.pop("COUNT")
    assert sorted(defs.values()) == list(range(count))
    assert len(b.PIPE_CLASSES) == count
    for name, idx in defs.items():
        assert b.PIPE_CLASSES[idx] == name.lower(), (name, idx)
    used = set(bench.class_counts(3, True)) | {"philox"}
    assert used <= set(b.PIPE_CLASSES) | {"alu", "ffma"}
