"""The C-ABI library loads and exports every function include/tdarisp.h declares
(no GPU needed: nothing here calls into CUDA)."""
from __future__ import annotations

import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tdarisp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(tr_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    return tdarisp.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("tr_create", "tr_set_molecule", "tr_set_orbitals", "tr_build", "tr_matvec",
              "tr_solve", "tr_last_error", "tr_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    from paper_2603_29257_gb300 import tdarisp
    assert set(declared_functions()) <= set(tdarisp.SIGNATURES)


def test_version_and_defaults(lib):
    from paper_2603_29257_gb300 import tdarisp
    assert lib.tr_version() >= 100
    o = tdarisp.default_options()
    assert o.cx == 0.25 and o.k_alpha == 1.0 and o.window_ev == 40.0 and o.aux_on_h == 0


def test_null_arguments_are_rejected_without_a_gpu(lib):
    from paper_2603_29257_gb300 import tdarisp
    assert lib.tr_create(None, None, None) == tdarisp.TR_EINVAL
    assert lib.tr_build(None) == tdarisp.TR_EINVAL
    assert lib.tr_build_batch(None, 0, 0) == tdarisp.TR_EINVAL
    assert lib.tr_matvec(None, 1, None, None, 0) == tdarisp.TR_EINVAL
    lib.tr_destroy(None)
    assert lib.tr_last_error(None) == b"null context"
