"""GB300 multi-reference alignment (MRA) of 2D particle images.

Thin Python binding of the C-ABI library ``libmra.so`` (see ``include/mra.h``):
argument marshalling only.  Every step of the alignment runs in the
library's CUDA kernels; torch supplies device memory and streams.  There is
no CPU fallback: importing works without a GPU, but every call needs the
built library and a CUDA device, and raises otherwise.

The functions carry the C names (``mra_create``, ``mra_set_refs``,
``mra_align``, ``mra_average``, ...); :class:`Aligner` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

__all__ = [
    "MRA_OK", "MRA_EINVAL", "MRA_ESTATE", "MRA_ENOMEM", "MRA_ECUDA", "MRA_ETIMEOUT", "MRA_EUNSUPPORTED",
    "MRA_FP32", "MRA_BF16_RESCORE", "MRA_FP16_RESCORE", "MRA_KERNEL_AUTO", "MRA_KERNEL_MMA_SYNC",
    "MRA_KERNEL_TCGEN05", "MRAError", "MRAConfig", "MRAInfo", "POSE_FIELDS",
    "library_path", "load_library", "mra_create", "mra_destroy", "mra_last_error", "mra_get_info",
    "mra_set_refs", "mra_align", "mra_average", "mra_class_sums", "mra_average_finalize", "mra_run_host",
    "mra_debug_polar", "mra_debug_spectra", "mra_debug_cc", "mra_profile", "mra_profile_read", "mra_sync",
    "mra_align_static", "mra_refresh_refs", "mra_copy_refs", "mra_run_graph", "mra_graph_info", "STAGES",
    "Aligner", "decode_poses", "EXPORTED_SYMBOLS",
]

MRA_OK, MRA_EINVAL, MRA_ESTATE, MRA_ENOMEM, MRA_ECUDA, MRA_ETIMEOUT, MRA_EUNSUPPORTED = range(7)
MRA_FP32, MRA_BF16_RESCORE, MRA_FP16_RESCORE = 0, 1, 2
MRA_KERNEL_AUTO, MRA_KERNEL_MMA_SYNC, MRA_KERNEL_TCGEN05 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))

EXPORTED_SYMBOLS = [
    "mra_create", "mra_destroy", "mra_last_error", "mra_get_info", "mra_set_refs", "mra_align",
    "mra_average", "mra_class_sums", "mra_average_finalize", "mra_run_host", "mra_debug_polar",
    "mra_debug_spectra", "mra_debug_cc", "mra_profile", "mra_profile_read", "mra_sync", "mra_align_static", "mra_refresh_refs",
    "mra_copy_refs", "mra_run_graph", "mra_graph_info",
]

STAGES = ("polar", "refs", "cc", "decode", "average", "rescore", "convert", "unused")

# mra_pose_t: int32 k, ang_idx, mirror, shift_idx; float32 angle_deg, sx, sy, cc
POSE_FIELDS = ("k", "ang_idx", "mirror", "shift_idx", "angle_deg", "sx", "sy", "cc")


class MRAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"MRA status {code}: {msg}")
        self.code = code


class MRAConfig(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("first_ring", ctypes.c_int32), ("last_ring", ctypes.c_int32),
                ("ring_step", ctypes.c_int32), ("shift_range", ctypes.c_float), ("shift_step", ctypes.c_float),
                ("mirror", ctypes.c_int32), ("precision", ctypes.c_int32), ("chunk_images", ctypes.c_int32),
                ("kernel", ctypes.c_int32)]


class MRAInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("n_rings", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("n_bins", ctypes.c_int32), ("n_bins_padded", ctypes.c_int32), ("S", ctypes.c_int32),
                ("K", ctypes.c_int32), ("chunk_images", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


class MRAStageTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


def library_path() -> str:
    return os.path.join(_HERE, "libmra.so")


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load ``libmra.so``; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "mra_create": ([ctypes.POINTER(MRAConfig), ctypes.POINTER(vp)], ctypes.c_int),
        "mra_destroy": ([vp], ctypes.c_int),
        "mra_last_error": ([vp], ctypes.c_char_p),
        "mra_get_info": ([vp, ctypes.POINTER(MRAInfo)], ctypes.c_int),
        "mra_set_refs": ([vp, vp, i32, vp], ctypes.c_int),
        "mra_copy_refs": ([vp, vp, vp], ctypes.c_int),
        "mra_align": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "mra_average": ([vp, vp, vp, i64, vp, vp, vp], ctypes.c_int),
        "mra_class_sums": ([vp, vp, vp, i64, vp, vp, vp, vp], ctypes.c_int),
        "mra_average_finalize": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "mra_run_host": ([vp, vp, i32, vp, i64, vp, vp, vp, vp], ctypes.c_int),
        "mra_debug_polar": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "mra_debug_spectra": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "mra_debug_cc": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "mra_profile": ([vp, ctypes.c_int], ctypes.c_int),
        "mra_sync": ([vp, vp], ctypes.c_int),
        "mra_refresh_refs": ([vp, vp, vp, i32, vp, vp, i64, vp], ctypes.c_int),
        "mra_align_static": ([ctypes.POINTER(MRAConfig), vp, i32, vp, i64, vp, vp, ctypes.c_char_p, i32],
                             ctypes.c_int),
        "mra_profile_read": ([vp, ctypes.POINTER(MRAStageTime)], ctypes.c_int),
        "mra_run_graph": ([vp, vp, i32, vp, i64, vp, vp, vp, vp], ctypes.c_int),
        "mra_graph_info": ([vp, ctypes.POINTER(i32)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(rc: int, h) -> None:
    if rc != MRA_OK:
        msg = load_library().mra_last_error(h)
        raise MRAError(rc, msg.decode() if msg else "")


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t: torch.Tensor, dtype, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check_stack(t: torch.Tensor, L: int, name: str) -> None:
    """A stack of L x L images: [n, L, L] (checked before any pointer reaches the library)."""
    if t.dim() != 3 or tuple(t.shape[1:]) != (L, L):
        raise ValueError(f"{name} must have shape [n, {L}, {L}], got {list(t.shape)}")


def _check_poses(p: torch.Tensor, n: int, name: str = "poses") -> None:
    if p.dim() != 2 or tuple(p.shape) != (n, 8):
        raise ValueError(f"{name} must have shape [{n}, 8] (mra_pose_t rows), got {list(p.shape)}")


def _host_ptr(a, dtype, name: str):
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous host {dtype} tensor")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"{name} must be a host torch tensor")


def mra_create(L: int, first_ring: int, last_ring: int, ring_step: int = 1, shift_range: float = 0.0,
               shift_step: float = 1.0, mirror: int = 1, precision: int = MRA_FP32, chunk_images: int = 0,
               kernel: int = MRA_KERNEL_AUTO):
    cfg = MRAConfig(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision, chunk_images,
                    kernel)
    h = ctypes.c_void_p()
    lib = load_library()
    rc = lib.mra_create(ctypes.byref(cfg), ctypes.byref(h))
    if rc != MRA_OK:
        raise MRAError(rc, (lib.mra_last_error(None) or b"").decode())
    return h


def mra_destroy(h) -> None:
    _check(load_library().mra_destroy(h), None)


def mra_last_error(h) -> str:
    return (load_library().mra_last_error(h) or b"").decode()


def mra_get_info(h) -> dict:
    info = MRAInfo()
    _check(load_library().mra_get_info(h, ctypes.byref(info)), h)
    return {f: getattr(info, f) for f, _ in MRAInfo._fields_}


def mra_set_refs(h, refs: torch.Tensor, stream=None) -> None:
    _check(load_library().mra_set_refs(h, _dev_ptr(refs, torch.float32, "refs"), refs.shape[0], _stream(stream)), h)


def mra_copy_refs(dst, src, stream=None) -> None:
    """Give handle ``dst`` the resident reference spectra of ``src`` (same configuration)."""
    _check(load_library().mra_copy_refs(dst, src, _stream(stream)), dst)


def mra_align(h, imgs: torch.Tensor, poses: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Returns poses as an int32 tensor [n, 8] in mra_pose_t layout (see :func:`decode_poses`)."""
    n = imgs.shape[0]
    if imgs.dim() != 3 or imgs.shape[1] != imgs.shape[2]:
        raise ValueError(f"imgs must have shape [n, L, L], got {list(imgs.shape)}")
    if poses is None:
        poses = torch.empty((n, 8), dtype=torch.int32, device=imgs.device)
    _check_poses(poses, n)
    _check(load_library().mra_align(h, _dev_ptr(imgs, torch.float32, "imgs"), n,
                                    _dev_ptr(poses, torch.int32, "poses"), _stream(stream)), h)
    return poses


def mra_average(h, imgs: torch.Tensor, poses: torch.Tensor, avg: torch.Tensor, counts: torch.Tensor,
                stream=None) -> None:
    _check(load_library().mra_average(h, _dev_ptr(imgs, torch.float32, "imgs"), _dev_ptr(poses, torch.int32, "poses"),
                                      imgs.shape[0], _dev_ptr(avg, torch.float32, "avg"),
                                      _dev_ptr(counts, torch.int32, "counts"), _stream(stream)), h)


def mra_class_sums(h, imgs, poses, sums, comp, counts, stream=None) -> None:
    _check(load_library().mra_class_sums(h, _dev_ptr(imgs, torch.float32, "imgs"),
                                         _dev_ptr(poses, torch.int32, "poses"), imgs.shape[0],
                                         _dev_ptr(sums, torch.float32, "sums"), _dev_ptr(comp, torch.float32, "comp"),
                                         _dev_ptr(counts, torch.int32, "counts"), _stream(stream)), h)


def mra_average_finalize(h, sums, comp, counts, avg, stream=None) -> None:
    _check(load_library().mra_average_finalize(h, _dev_ptr(sums, torch.float32, "sums"),
                                               _dev_ptr(comp, torch.float32, "comp"),
                                               _dev_ptr(counts, torch.int32, "counts"),
                                               _dev_ptr(avg, torch.float32, "avg"), _stream(stream)), h)


def mra_run_host(h, refs: torch.Tensor, imgs: torch.Tensor, poses: torch.Tensor, avg: torch.Tensor,
                 counts: torch.Tensor, stream=None) -> None:
    """Whole pass from host tensors (pinned memory recommended); synchronous."""
    _check(load_library().mra_run_host(h, _host_ptr(refs, torch.float32, "refs"), refs.shape[0],
                                       _host_ptr(imgs, torch.float32, "imgs"), imgs.shape[0],
                                       _host_ptr(poses, torch.int32, "poses"), _host_ptr(avg, torch.float32, "avg"),
                                       _host_ptr(counts, torch.int32, "counts"), _stream(stream)), h)


def _debug(fn_name, h, imgs, out, stream):
    fn = getattr(load_library(), fn_name)
    _check(fn(h, _dev_ptr(imgs, torch.float32, "imgs"), imgs.shape[0], _dev_ptr(out, torch.float32, "out"),
              _stream(stream)), h)
    return out


def mra_debug_polar(h, imgs, out, stream=None):
    return _debug("mra_debug_polar", h, imgs, out, stream)


def mra_debug_spectra(h, imgs, out, stream=None):
    return _debug("mra_debug_spectra", h, imgs, out, stream)


def mra_debug_cc(h, imgs, out, stream=None):
    return _debug("mra_debug_cc", h, imgs, out, stream)


def mra_sync(h, stream=None) -> None:
    """Wait for the handle's work on the stream; raises MRAError(MRA_ETIMEOUT) after a device time-out."""
    _check(load_library().mra_sync(h, _stream(stream)), h)


def mra_refresh_refs(h, refs: torch.Tensor, counts: torch.Tensor, reseed: Optional[torch.Tensor] = None,
                     imgs: Optional[torch.Tensor] = None, stream=None) -> None:
    """Normalise populated classes (and reseed empty ones from chosen images) in place; see include/mra.h."""
    rs = _dev_ptr(reseed, torch.int32, "reseed") if reseed is not None else None
    im = _dev_ptr(imgs, torch.float32, "imgs") if imgs is not None else None
    n = imgs.shape[0] if imgs is not None else 0
    _check(load_library().mra_refresh_refs(h, _dev_ptr(refs, torch.float32, "refs"),
                                           _dev_ptr(counts, torch.int32, "counts"), refs.shape[0], rs, im, n,
                                           _stream(stream)), h)


def mra_align_static(refs: torch.Tensor, imgs: torch.Tensor, poses: torch.Tensor, L: int, first_ring: int,
                     last_ring: int, ring_step: int = 1, shift_range: float = 0.0, shift_step: float = 1.0,
                     mirror: int = 1, stream=None) -> None:
    """FP32 alignment that allocates no device memory (no handle); see include/mra.h."""
    _check_stack(refs, L, "refs")
    _check_stack(imgs, L, "imgs")
    _check_poses(poses, imgs.shape[0])
    cfg = MRAConfig(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, MRA_FP32, 0, 0)
    buf = ctypes.create_string_buffer(512)
    rc = load_library().mra_align_static(ctypes.byref(cfg), _dev_ptr(refs, torch.float32, "refs"), refs.shape[0],
                                         _dev_ptr(imgs, torch.float32, "imgs"), imgs.shape[0],
                                         _dev_ptr(poses, torch.int32, "poses"), _stream(stream), buf, len(buf))
    if rc != MRA_OK:
        raise MRAError(rc, buf.value.decode())


def mra_run_graph(h, refs: torch.Tensor, imgs: torch.Tensor, poses: torch.Tensor, avg: torch.Tensor,
                  counts: torch.Tensor, stream=None) -> None:
    """set_refs + align + class average as one cached CUDA graph launch (see include/mra.h)."""
    if imgs.dim() != 3 or refs.dim() != 3 or tuple(refs.shape[1:]) != tuple(imgs.shape[1:]):
        raise ValueError(f"refs {list(refs.shape)} and imgs {list(imgs.shape)} must be stacks of one box size")
    _check_poses(poses, imgs.shape[0])
    if tuple(avg.shape) != tuple(refs.shape) or tuple(counts.shape) != (refs.shape[0],):
        raise ValueError("avg must match refs and counts must have one entry per reference")
    _check(load_library().mra_run_graph(h, _dev_ptr(refs, torch.float32, "refs"), refs.shape[0],
                                        _dev_ptr(imgs, torch.float32, "imgs"), imgs.shape[0],
                                        _dev_ptr(poses, torch.int32, "poses"), _dev_ptr(avg, torch.float32, "avg"),
                                        _dev_ptr(counts, torch.int32, "counts"), _stream(stream)), h)


def mra_graph_info(h) -> bool:
    """True once mra_run_graph holds an instantiated graph for the handle."""
    v = ctypes.c_int32()
    _check(load_library().mra_graph_info(h, ctypes.byref(v)), h)
    return bool(v.value)


def mra_profile(h, enable: bool) -> None:
    """Turn per-stage CUDA-event timing on/off (clears the counters)."""
    _check(load_library().mra_profile(h, 1 if enable else 0), h)


def mra_profile_read(h) -> dict:
    """Per-stage {launches, ms} since the last mra_profile call (waits for the events)."""
    arr = (MRAStageTime * len(STAGES))()
    _check(load_library().mra_profile_read(h, arr), h)
    return {name: {"launches": int(arr[i].launches), "ms": float(arr[i].ms)} for i, name in enumerate(STAGES)}


def decode_poses(poses: torch.Tensor) -> dict:
    """mra_pose_t rows (int32 [n, 8]) -> dict of numpy arrays."""
    p = poses.detach().cpu().contiguous()
    ints = p.numpy()
    flts = p.view(torch.float32).numpy()
    return {"k": ints[:, 0].copy(), "ang_idx": ints[:, 1].copy(), "mirror": ints[:, 2].copy(),
            "shift_idx": ints[:, 3].copy(), "angle_deg": flts[:, 4].copy(), "sx": flts[:, 5].copy(),
            "sy": flts[:, 6].copy(), "cc": flts[:, 7].copy()}


class Aligner:
    """Owns one library handle: references resident on the device, workspace reused."""

    def __init__(self, L, first_ring, last_ring, ring_step=1, shift_range=0.0, shift_step=1.0, mirror=1,
                 precision=MRA_FP32, chunk_images=0, kernel=MRA_KERNEL_AUTO):
        self.L = L
        self.h = mra_create(L, first_ring, last_ring, ring_step, shift_range, shift_step, mirror, precision,
                            chunk_images, kernel)
        self.K = 0

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            mra_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return mra_get_info(self.h)

    def set_refs(self, refs: torch.Tensor, stream=None):
        _check_stack(refs, self.L, "refs")
        mra_set_refs(self.h, refs, stream)
        self.K = refs.shape[0]

    def copy_refs(self, other: "Aligner", stream=None):
        mra_copy_refs(self.h, other.h, stream)
        self.K = other.K

    def align(self, imgs: torch.Tensor, poses=None, stream=None) -> torch.Tensor:
        _check_stack(imgs, self.L, "imgs")
        if poses is not None:
            _check_poses(poses, imgs.shape[0])
        return mra_align(self.h, imgs, poses, stream)

    def average(self, imgs, poses, avg=None, counts=None, stream=None):
        _check_stack(imgs, self.L, "imgs")
        _check_poses(poses, imgs.shape[0])
        if avg is not None:
            _check_stack(avg, self.L, "avg")
            if avg.shape[0] != self.K:
                raise ValueError(f"avg must hold K = {self.K} classes, got {avg.shape[0]}")
        if counts is not None and tuple(counts.shape) != (self.K,):
            raise ValueError(f"counts must have shape [{self.K}], got {list(counts.shape)}")
        if avg is None:
            avg = torch.zeros((self.K, self.L, self.L), dtype=torch.float32, device=imgs.device)
        if counts is None:
            counts = torch.empty((self.K,), dtype=torch.int32, device=imgs.device)
        mra_average(self.h, imgs, poses, avg, counts, stream)
        return avg, counts

    def debug_polar(self, imgs, stream=None):
        _check_stack(imgs, self.L, "imgs")
        i = self.info
        out = torch.empty((imgs.shape[0], i["S"], i["n_samples"]), dtype=torch.float32, device=imgs.device)
        return mra_debug_polar(self.h, imgs, out, stream)

    def debug_spectra(self, imgs, stream=None):
        _check_stack(imgs, self.L, "imgs")
        i = self.info
        out = torch.empty((imgs.shape[0], i["S"], i["n_bins"], 2), dtype=torch.float32, device=imgs.device)
        return mra_debug_spectra(self.h, imgs, out, stream)

    def debug_cc(self, imgs, stream=None):
        _check_stack(imgs, self.L, "imgs")
        i = self.info
        out = torch.empty((imgs.shape[0], self.K, i["S"], 2, i["M"]), dtype=torch.float32, device=imgs.device)
        return mra_debug_cc(self.h, imgs, out, stream)
