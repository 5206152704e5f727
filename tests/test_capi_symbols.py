"""The C-ABI library loads without a GPU and exports every entry point that
include/mm.h declares; argument validation that needs no device works."""

import ctypes
import os
import re

import pytest

import paper_2606_01114_gb300 as mm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2606_01114_gb300 import build
    build.build()
    return mm._load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mm_init_mesh", "mm_set_material", "mm_demag_field", "mm_exchange_field",
                     "mm_llg_step", "mm_relax", "mm_energy", "mm_destroy", "mm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_python_binding_has_the_same_names(lib):
    for name in declared_functions():
        assert callable(getattr(mm, name)), name


@pytest.mark.parametrize("n", [(4, 4, 6), (4, 0, 4), (1024, 4, 4), (4, 4, 3), (513, 8, 1)])
def test_invalid_mesh_rejected_without_device_work(lib, n):
    with pytest.raises(mm.MMError) as e:
        mm.mm_init_mesh(*n, 1e-9, 1e-9, 1e-9)
    assert e.value.code == mm.MM_ERR_INVALID_ARG


def test_invalid_spacing_and_precision(lib):
    with pytest.raises(mm.MMError) as e:
        mm.mm_init_mesh(4, 4, 4, -1e-9, 1e-9, 1e-9)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    with pytest.raises(mm.MMError) as e:
        mm.mm_init_mesh(4, 4, 4, 1e-9, 1e-9, 1e-9, precision=7)
    assert e.value.code == mm.MM_ERR_INVALID_ARG


def test_null_context_calls_fail_cleanly(lib):
    assert lib.mm_demag_field(None, None, None) == mm.MM_ERR_INVALID_ARG
    assert lib.mm_relax(None, None, 1.0, 1.0, 1, None, None) == mm.MM_ERR_INVALID_ARG
    lib.mm_destroy(None)
    assert lib.mm_kernel_launches(None) == 0
