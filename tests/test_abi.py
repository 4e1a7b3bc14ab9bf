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
    assert ctypes.sizeof(mra.MRAConfig) == 40
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
    (dict(L=32, first_ring=1, last_ring=5, kernel=3), "kernel"),
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


@pytest.mark.parametrize("precision", [mra.MRA_BF16_RESCORE, mra.MRA_FP16_RESCORE])
def test_create_rejects_configs_beyond_shared_memory(lib, precision):
    # L = 192 with rings 1..81: the polar kernel's CTA (the image in its zero
    # border, a row's ring samples and its 16-bit spectrum words) would need
    # about 350 KB of shared memory; the rescore CTA (image and ring samples,
    # spectra in place) would need about 260 KB
    with pytest.raises(mra.MRAError) as ei:
        mra.mra_create(L=192, first_ring=1, last_ring=81, shift_range=1.0, shift_step=1.0, precision=precision)
    assert ei.value.code == mra.MRA_EUNSUPPORTED
    assert "kernel would need" in str(ei.value) and "shared memory" in str(ei.value)


# Every configuration the GPU tests, the bench and the tools create.
_USED = [
    (76, 1, 35, 1, 4.0, 1.0), (76, 1, 35, 1, 2.0, 1.0), (76, 1, 35, 1, 3.0, 1.0),   # L = 76 workloads
    (128, 1, 60, 1, 6.0, 1.0), (128, 1, 60, 1, 1.0, 1.0),                            # L = 128 workload, parity case
    (132, 1, 65, 1, 1.0, 1.0),                                                       # rings beyond 64 at L = 132
    (90, 1, 36, 1, 6.0, 1.0), (90, 1, 36, 1, 1.0, 1.0),                              # RFA sweep
    (64, 1, 28, 1, 3.0, 1.0), (96, 1, 44, 1, 3.0, 1.0), (128, 1, 60, 1, 3.0, 1.0),   # serving boxes
    (32, 1, 12, 1, 1.5, 0.5), (48, 2, 20, 2, 2.0, 1.0), (24, 1, 15, 1, 2.0, 1.0),    # parity cases
    (16, 1, 2, 1, 1.0, 1.0), (16, 1, 4, 1, 1.0, 1.0), (20, 1, 6, 1, 2.0, 1.0),
    (48, 1, 22, 1, 1.0, 1.0), (32, 1, 12, 1, 2.0, 1.0), (40, 1, 16, 1, 2.0, 1.0), (48, 2, 16, 1, 2.0, 1.0),
    (48, 2, 18, 1, 1.0, 1.0), (32, 1, 10, 1, 1.0, 1.0), (32, 1, 10, 1, 0.0, 1.0),
]


@pytest.mark.parametrize("precision", [mra.MRA_FP32, mra.MRA_BF16_RESCORE, mra.MRA_FP16_RESCORE])
@pytest.mark.parametrize("cfg", _USED)
def test_used_configs_pass_the_shared_memory_check(lib, cfg, precision):
    L, r1, r2, dr, R, step = cfg
    try:
        h = mra.mra_create(L=L, first_ring=r1, last_ring=r2, ring_step=dr, shift_range=R, shift_step=step,
                           precision=precision)
    except mra.MRAError as e:  # no GPU here: the check passed and the first CUDA call failed
        assert e.code == mra.MRA_ECUDA, str(e)
    else:
        lib.mra_destroy(h)


def _static_call(lib, **kw):
    """mra_align_static with NULL buffers: only the checks before any CUDA call can run."""
    base = dict(L=32, first_ring=1, last_ring=5, ring_step=1, shift_range=1.0, shift_step=1.0, mirror=1,
                precision=mra.MRA_FP32, chunk_images=0, kernel=0)
    base.update(kw)
    cfg = mra.MRAConfig(*(base[f] for f, _ in mra.MRAConfig._fields_))
    buf = ctypes.create_string_buffer(512)
    rc = lib.mra_align_static(ctypes.byref(cfg), None, 3, None, 0, None, None, buf, len(buf))
    return rc, buf.value.decode()


@pytest.mark.parametrize("kw,code,needle", [
    # 50001 x 50001 shifts: the grid size must be checked without integer overflow
    (dict(shift_range=25000.0, shift_step=1.0), mra.MRA_EINVAL, "4096"),
    (dict(shift_range=float("inf"), shift_step=1.0), mra.MRA_EINVAL, "shift_range"),
    (dict(shift_range=1.0, shift_step=float("inf")), mra.MRA_EINVAL, "shift_step"),
    (dict(shift_range=float("nan")), mra.MRA_EINVAL, "shift_range"),
    (dict(last_ring=90), mra.MRA_EINVAL, "M = 1024"),
    (dict(L=31), mra.MRA_EINVAL, "L must be even"),
    # the same shared-memory admission as mra_create (the FP32 contraction CTA of M = 512 fits; a
    # 1024-pixel box does not fit the polar kernel's staged image)
    (dict(L=1024, first_ring=1, last_ring=60), mra.MRA_EUNSUPPORTED, "shared memory"),
    (dict(precision=mra.MRA_BF16_RESCORE), mra.MRA_EUNSUPPORTED, "FP32 path only"),
])
def test_static_entry_checks_the_configuration_like_create(lib, kw, code, needle):
    rc, msg = _static_call(lib, **kw)
    assert rc == code, msg
    assert needle in msg, msg


def test_static_entry_and_create_agree_on_every_rejection(lib):
    for kw in (dict(shift_range=25000.0), dict(shift_range=float("inf")), dict(L=1024, last_ring=60),
               dict(ring_step=0), dict(mirror=3)):
        rc, msg = _static_call(lib, **kw)
        cfg = dict(L=32, first_ring=1, last_ring=5, shift_range=1.0, shift_step=1.0)
        cfg.update(kw)
        with pytest.raises(mra.MRAError) as ei:
            mra.mra_create(**cfg)
        assert ei.value.code == rc and str(ei.value).endswith(msg), (kw, rc, msg, str(ei.value))
