"""The C-ABI library builds and exports every entry point of include/*.h
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

from paper_1701_03038_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"FST_API\s+(?:const\s+)?\w+\s*\*?\s*(fst_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    assert {"fst_create", "fst_destroy", "fst_viterbi", "fst_forward_backward", "fst_viterbi_batch",
            "fst_forward_backward_batch", "fst_last_error"} <= names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in sorted(declared_symbols()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    names = declared_symbols()
    bound = set(_lib.SIGNATURES) | {"fst_last_error"}
    assert names <= bound, names - bound


def test_library_does_not_link_libtorch(libpath):
    data = open(libpath, "rb").read()
    assert b"libtorch" not in data and b"libc10" not in data


def test_last_error_callable_without_gpu(libpath):
    lib = _lib.load()
    assert lib.fst_last_error() is not None


def test_invalid_args_rejected_without_gpu(libpath):
    lib = _lib.load()
    out = ctypes.c_void_p()
    # Q = 0 is rejected before any CUDA call
    rc = lib.fst_create(0, 0, None, None, None, None, None, 0, None, None, 1, 0, ctypes.byref(out))
    assert rc == _lib.INVALID_ARG and not out.value
    assert b"bad sizes" in lib.fst_last_error()


def test_debug_checks_unsupported_in_a_normal_build(libpath):
    # the bounds-checked record exists only in a -DFST_DEBUG build; a normal
    # build says so (no device call is made)
    lib = _lib.load()
    v = ctypes.c_int64(-1)
    rc = lib.fst_debug_checks(ctypes.byref(v), None, None, None)
    assert rc == _lib.UNSUPPORTED and v.value == -1
    assert b"FST_DEBUG" in lib.fst_last_error()


def test_every_declaration_cites_its_passage():
    # each entry point's comment cites the paper passage it follows (a
    # section, algorithm, equation, figure or table) or says the paper has
    # no counterpart
    h = open(os.path.join(ROOT, "include", "fstgpu.h")).read()
    decls = list(re.finditer(r"FST_API[^;]*?\b(fst_[a-z0-9_]+)\s*\(", h))
    assert len(decls) > 40
    prev, missing = 0, []
    for m in decls:
        if not re.search(r"Sec\.|Alg\.|Eq\.|Fig\.|Table|paper", h[prev:m.start()]):
            missing.append(m.group(1))
        prev = m.end()
    assert not missing, missing
