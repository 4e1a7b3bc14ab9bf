"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

No compute call runs here (no GPU); argument validation that happens before
any CUDA call is exercised.
"""
import ctypes
import os
import re

import pytest

import __graft_entry__ as entry
import paper_2011_05755_gb300 as mra

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return mra.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "mra.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mra_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mra_create", "mra_set_refs", "mra_align", "mra_average", "mra_destroy", "mra_last_error"]:
        assert n in names
    assert sorted(mra.EXPORTED_SYMBOLS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(mra.MRAConfig) == 36
    assert ctypes.sizeof(mra.MRAInfo) == 40
    assert len(mra.POSE_FIELDS) == 8  # mra_pose_t is 8 x 4 bytes


@pytest.mark.parametrize("kw,needle", [
    (dict(L=31, first_ring=1, last_ring=5), "L must be even"),
    (dict(L=32, first_ring=0, last_ring=5), "first_ring"),
    (dict(L=32, first_ring=5, last_ring=4), "last_ring"),
    (dict(L=32, first_ring=1, last_ring=5, ring_step=0), "ring_step"),
    (dict(L=32, first_ring=1, last_ring=5, shift_range=1.0, shift_step=0.0), "shift_step"),
    (dict(L=32, first_ring=1, last_ring=5, shift_range=1.0, shift_step=0.75), "integer"),
    (dict(L=32, first_ring=1, last_ring=5, shift_range=40.0, shift_step=1.0), "4096"),
    (dict(L=32, first_ring=1, last_ring=5, mirror=2), "mirror"),
    (dict(L=32, first_ring=1, last_ring=5, precision=7), "precision"),
])
def test_create_rejects_bad_config_before_touching_cuda(lib, kw, needle):
    with pytest.raises(mra.MRAError) as ei:
        mra.mra_create(**kw)
    assert ei.value.code == mra.MRA_EINVAL
    assert needle in str(ei.value)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.mra_destroy(None) == mra.MRA_OK
    assert lib.mra_align(None, None, 0, None, None) == mra.MRA_EINVAL
    assert b"handle is NULL" in lib.mra_last_error(None)
