"""The C-ABI library builds for sm_103a, loads, and exports every function
include/libmemsynth.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mem_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1703_02920_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["mem_create", "mem_forward", "mem_adjoint", "mem_objective_grad", "mem_solve", "mem_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_names_match_the_abi():
    from paper_1703_02920_gb300 import memsynth
    for name in _declared():
        if name in ("mem_status_string", "mem_last_error", "mem_num_vis", "mem_num_images",
                    "mem_scalars_dev"):
            continue
        assert hasattr(memsynth, name), name


def test_status_strings_without_gpu(lib):
    lib.mem_status_string.restype = ctypes.c_char_p
    assert lib.mem_status_string(0) == b"ok"
    assert lib.mem_status_string(4) == b"device wait timed out"


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Argument validation happens on the host before any CUDA call."""
    from paper_1703_02920_gb300 import memsynth as ms
    ms.load()
    import numpy as np
    offs = np.array([0, 3], dtype=np.int64)
    u = np.zeros(3); v = np.zeros(3); vo = np.zeros(6); pb = np.ones((1, 32, 32), np.float32)
    with pytest.raises(ms.MemError) as e:
        ms.mem_create(30, 1e-6, 1e-6, offs, 0.0, 1e-4, 0, 0, u, v, vo, np.ones(3), pb)   # N not multiple of 16
    assert e.value.status == 1
    with pytest.raises(ms.MemError) as e:
        ms.mem_create(32, 1e-6, 1e-6, offs, 0.0, 1e-4, 0, 0, u, v, vo, np.array([1.0, 0.0, 1.0]), pb)
    assert e.value.status == 1   # sigma must be > 0
    with pytest.raises(ms.MemError) as e:
        ms.mem_create(32, 1e-6, 1e-6, offs, 0.0, -1.0, 0, 0, u, v, vo, np.ones(3), pb)
    assert e.value.status == 1   # G must be > 0
    with pytest.raises(ms.MemError) as e:
        ms.mem_create(96, 1e-6, 1e-6, offs, 0.0, 1e-4, 2, 0, u, v, vo, np.ones(3), np.ones((1, 96, 96), np.float32))
    assert e.value.status == 6   # tensor-core form shape


def test_every_declaration_is_documented():
    """Each function the header declares sits in a block (lines between blank
    lines) that opens with its comment: the passage it implements, argument
    layout, ownership, errors; one comment may cover a group of related
    declarations."""
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        for block in re.split(r"\n\s*\n", src):
            decl = re.search(r"^[A-Za-z_][A-Za-z0-9_ \*]*\b(mem_[a-z0-9_]+)\s*\(", block, flags=re.M)
            if decl and not block.lstrip().startswith(("/*", "#", "typedef", "}")):
                raise AssertionError((fn, decl.group(1)))
            if decl and block.lstrip().startswith(("#", "typedef", "}")):
                # a declaration inside a larger construct: its own comment must precede it
                assert block[:decl.start()].rstrip().endswith("*/"), (fn, decl.group(1))
