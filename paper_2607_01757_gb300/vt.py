"""Thin ctypes binding of libvt (include/vt.h).

Argument marshalling only: every step of the tracking path runs in the CUDA
library.  Functions carry the C names; tensors are torch tensors on the GPU
(their ``data_ptr``), images may also be host numpy / CPU torch arrays for the
``vt_pyramid_build*`` calls.  There is no CPU fallback: importing this module
raises if libvt.so cannot be loaded.
"""

from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass

from . import build as _build

VT_OK, VT_ERR_ARG, VT_ERR_OOM, VT_ERR_CUDA, VT_ERR_TIMEOUT, VT_ERR_UNSUPPORTED = range(6)
VT_GRAD_NONE, VT_GRAD_S16, VT_GRAD_F16 = 0, 1, 2
VT_TRACKED, VT_LOST_EIG, VT_LOST_OOB, VT_LOST_FB, VT_LOST_INPUT = range(5)
VT_MAX_LEVELS = 8
VT_DEFAULT_MIN_EIG = 1e-4
SUPPORTED_WINDOWS = (9, 15, 21, 31)


class VTError(RuntimeError):
    def __init__(self, what: str, code: int):
        super().__init__(f"{what}: {vt_status_str(code)}")
        self.code = code


def _load() -> C.CDLL:
    override = os.environ.get("VT_LIBRARY")
    if override:  # an explicitly chosen build of libvt.so
        return C.CDLL(override)
    path = _build.LIB
    if not os.path.exists(path) or _build.needs_build():
        try:
            path = _build.build()
        except Exception as e:  # noqa: BLE001 - report why the library is unusable
            raise ImportError(f"libvt.so is missing and could not be built ({e}); "
                              "build it with: python -m paper_2607_01757_gb300.build") from e
    return C.CDLL(path)


_lib = _load()
LIB_PATH = _lib._name

vp, i32, f32 = C.c_void_p, C.c_int, C.c_float


class vt_klt_params(C.Structure):
    _fields_ = [("win", i32), ("levels", i32), ("max_iters", i32), ("eps", f32), ("min_eig", f32),
                ("fb_thr", f32)]


class vt_klt_diag(C.Structure):
    _fields_ = [("reason", vp), ("iters", vp), ("lmin", vp), ("flops", vp), ("sweeps", vp)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("vt_pyramid_build", i32, [vp, i32, i32, i32, i32, i32, vp, C.POINTER(vp)])
_sig("vt_pyramid_build_grad", i32, [vp, i32, i32, i32, i32, i32, i32, vp, C.POINTER(vp)])
_sig("vt_gradients", i32, [vp, i32, vp])
_sig("vt_pyramid_level", i32, [vp, i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)])
_sig("vt_pyramid_grad", i32, [vp, i32, C.POINTER(vp), C.POINTER(i32), C.POINTER(i32)])
_sig("vt_pyramid_info", i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_size_t)])
_sig("vt_pyramid_free", None, [vp])
_sig("vt_klt_track", i32, [vp, vp, vp, i32, vp, i32, i32, i32, f32, vp, vp, vp, vp])
_sig("vt_klt_track_ex", i32, [vp, vp, vp, i32, vp, C.POINTER(vt_klt_params), vp, vp, vp,
                              C.POINTER(vt_klt_diag), vp])
_sig("vt_klt_track_fb", i32, [vp, vp, vp, i32, C.POINTER(vt_klt_params), vp, vp, vp, C.POINTER(vt_klt_diag), vp])
_sig("vt_fb_check", i32, [vp, vp, vp, vp, i32, f32, vp, vp])
_sig("vt_pyramid_create", i32, [i32, i32, i32, C.POINTER(vp)])
_sig("vt_pyramid_create_on", i32, [vp, i32, C.c_size_t, i32, i32, i32, C.POINTER(vp)])
_sig("vt_status_str", C.c_char_p, [i32])
_sig("vt_version", C.c_char_p, [])


def header_functions() -> list:
    """Names of every function declared in include/vt.h."""
    with open(os.path.join(_build.INCLUDE, "vt.h")) as f:
        text = f.read()
    return re.findall(r"^VT_API\s+[\w\s\*]*?\b(vt_\w+)\s*\(", text, flags=re.M)


# ------------------------------------------------------------------ marshalling
def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(code, what):
    if code != VT_OK:
        raise VTError(what, code)


def vt_status_str(code: int) -> str:
    return _lib.vt_status_str(code).decode()


def vt_version() -> str:
    return _lib.vt_version().decode()


_sig("vt_fp32_fma_probe", i32, [i32, vp, C.c_longlong, C.POINTER(C.c_longlong), vp])


def vt_fp32_fma_probe(iters: int, out, stream=None) -> int:
    """Launch the FP32 FMA throughput probe (a measurement helper); returns
    the launch's FLOP count.  ``out``: device float32 tensor of at least
    SMs x 2048 entries."""
    fl = C.c_longlong()
    _check(_lib.vt_fp32_fma_probe(int(iters), _ptr(out), int(out.numel()), C.byref(fl), _stream(stream)),
           "vt_fp32_fma_probe")
    return int(fl.value)


class Pyramid:
    """Owning handle of a library pyramid (vt_pyramid*)."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)

    def free(self):
        if self.handle:
            _lib.vt_pyramid_free(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def info(self):
        return vt_pyramid_info(self)

    def level(self, lvl: int):
        """Zero-copy torch view (uint8 [h, w], row stride = pitch) of level lvl."""
        ptr, w, h, pitch = vt_pyramid_level(self, lvl)
        return _device_view(ptr, (h, w), (pitch, 1), "|u1")

    def grad(self, lvl: int):
        """Zero-copy view of level lvl's gradient pairs: int16 [h, w, 2] for
        S16, float16 [h, w, 2] for F16."""
        ptr, gpitch, t = vt_pyramid_grad(self, lvl)
        _, w, h, _ = vt_pyramid_level(self, lvl)
        typestr = "<i2" if t == VT_GRAD_S16 else "<f2"
        if t == VT_GRAD_NONE:
            raise ValueError("pyramid has no gradients")
        return _device_view(ptr, (h, w, 2), (gpitch * 4, 4, 2), typestr)


class _CAI:
    def __init__(self, ptr, shape, strides, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "strides": strides, "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def _device_view(ptr, shape, strides, typestr):
    import torch

    return torch.as_tensor(_CAI(ptr, shape, strides, typestr), device="cuda")


def _img_args(img):
    """(pointer, w, h, pitch, on_device) of a 2-D uint8 image."""
    if hasattr(img, "data_ptr"):  # torch
        if img.dtype.itemsize != 1 or img.dim() != 2 or img.stride(1) != 1:
            raise ValueError("image must be a 2-D uint8 tensor with unit column stride")
        return img.data_ptr(), img.shape[1], img.shape[0], img.stride(0), int(img.is_cuda)
    import numpy as np

    a = img
    if a.dtype != np.uint8 or a.ndim != 2 or a.strides[1] != 1:
        raise ValueError("image must be a 2-D uint8 array with unit column stride")
    return a.ctypes.data, a.shape[1], a.shape[0], a.strides[0], 0


def vt_pyramid_build(img, levels: int, stream=None, out: Pyramid | None = None) -> Pyramid:
    p, w, h, pitch, dev = _img_args(img)
    hd = C.c_void_p(out.handle if out is not None else None)
    _check(_lib.vt_pyramid_build(p, w, h, pitch, levels, dev, _stream(stream), C.byref(hd)), "vt_pyramid_build")
    return out if out is not None else Pyramid(hd.value)


def vt_pyramid_build_grad(img, levels: int, grad_type: int = VT_GRAD_S16, stream=None,
                          out: Pyramid | None = None) -> Pyramid:
    p, w, h, pitch, dev = _img_args(img)
    hd = C.c_void_p(out.handle if out is not None else None)
    _check(_lib.vt_pyramid_build_grad(p, w, h, pitch, levels, dev, grad_type, _stream(stream), C.byref(hd)),
           "vt_pyramid_build_grad")
    return out if out is not None else Pyramid(hd.value)


_sig("vt_pyramid_upload", i32, [vp, vp, i32, i32, vp])


def vt_pyramid_upload(pyr: Pyramid, img, stream=None) -> None:
    """Copy a frame (host or device array, the pyramid's w x h) into level 0
    of ``pyr``; a build that then names level 0 as its image copies nothing."""
    p, w, h, pitch, dev = _img_args(img)
    _check(_lib.vt_pyramid_upload(pyr, p, pitch, dev, _stream(stream)), "vt_pyramid_upload")


def vt_gradients(pyr: Pyramid, grad_type: int = VT_GRAD_S16, stream=None) -> None:
    _check(_lib.vt_gradients(pyr, grad_type, _stream(stream)), "vt_gradients")


def vt_pyramid_level(pyr: Pyramid, lvl: int):
    ptr, w, h, pitch = vp(), i32(), i32(), i32()
    _check(_lib.vt_pyramid_level(pyr, lvl, C.byref(ptr), C.byref(w), C.byref(h), C.byref(pitch)),
           "vt_pyramid_level")
    return ptr.value, w.value, h.value, pitch.value


def vt_pyramid_grad(pyr: Pyramid, lvl: int):
    ptr, gp, t = vp(), i32(), i32()
    _check(_lib.vt_pyramid_grad(pyr, lvl, C.byref(ptr), C.byref(gp), C.byref(t)), "vt_pyramid_grad")
    return ptr.value, gp.value, t.value


def vt_pyramid_info(pyr: Pyramid):
    w, h, L, b = i32(), i32(), i32(), C.c_size_t()
    _check(_lib.vt_pyramid_info(pyr, C.byref(w), C.byref(h), C.byref(L), C.byref(b)), "vt_pyramid_info")
    return w.value, h.value, L.value, b.value


def vt_pyramid_free(pyr: Pyramid) -> None:
    pyr.free()


@dataclass
class KltParams:
    win: int = 21
    levels: int = 4
    max_iters: int = 30
    eps: float = 0.01
    min_eig: float = VT_DEFAULT_MIN_EIG
    fb_thr: float = 0.5

    def c(self) -> vt_klt_params:
        return vt_klt_params(self.win, self.levels, self.max_iters, self.eps, self.min_eig, self.fb_thr)


def _diag(reason=None, iters=None, lmin=None, flops=None, sweeps=None):
    if reason is None and iters is None and lmin is None and flops is None and sweeps is None:
        return None
    return C.byref(vt_klt_diag(_ptr(reason), _ptr(iters), _ptr(lmin), _ptr(flops), _ptr(sweeps)))


def vt_klt_track(prev: Pyramid, cur: Pyramid, pts_in, pts_out, status, err=None, pts_guess=None, win=21,
                 levels=4, max_iters=30, eps=0.01, stream=None) -> None:
    n = int(pts_in.shape[0])
    _check(_lib.vt_klt_track(prev, cur, _ptr(pts_in), n, _ptr(pts_guess), win, levels, max_iters, eps,
                             _ptr(pts_out), _ptr(status), _ptr(err), _stream(stream)), "vt_klt_track")


def vt_klt_track_ex(prev: Pyramid, cur: Pyramid, pts_in, params: KltParams, pts_out, status, err=None,
                    pts_guess=None, reason=None, iters=None, lmin=None, flops=None, sweeps=None,
                    stream=None) -> None:
    n = int(pts_in.shape[0])
    prm = params.c()
    _check(_lib.vt_klt_track_ex(prev, cur, _ptr(pts_in), n, _ptr(pts_guess), C.byref(prm), _ptr(pts_out),
                                _ptr(status), _ptr(err), _diag(reason, iters, lmin, flops, sweeps),
                                _stream(stream)),
           "vt_klt_track_ex")


def vt_klt_track_fb(prev: Pyramid, cur: Pyramid, pts_in, params: KltParams, pts_out, status, err=None,
                    reason=None, iters=None, lmin=None, flops=None, sweeps=None, stream=None) -> None:
    n = int(pts_in.shape[0])
    prm = params.c()
    _check(_lib.vt_klt_track_fb(prev, cur, _ptr(pts_in), n, C.byref(prm), _ptr(pts_out), _ptr(status),
                                _ptr(err), _diag(reason, iters, lmin, flops, sweeps), _stream(stream)),
           "vt_klt_track_fb")


def vt_fb_check(p0, p0_back, st_f, st_b, thr, status_out, stream=None) -> None:
    n = int(p0.shape[0])
    _check(_lib.vt_fb_check(_ptr(p0), _ptr(p0_back), _ptr(st_f), _ptr(st_b), n, thr, _ptr(status_out),
                            _stream(stream)), "vt_fb_check")


def vt_pyramid_create(w: int, h: int, levels: int) -> Pyramid:
    hd = vp()
    _check(_lib.vt_pyramid_create(w, h, levels, C.byref(hd)), "vt_pyramid_create")
    return Pyramid(hd.value)


def vt_pyramid_create_on(level0, levels: int, nbytes: int | None = None) -> Pyramid:
    """A pyramid whose level 0 is the caller's device image `level0` (2-D
    uint8 CUDA tensor, rows 16-byte aligned; usually a view into a larger
    buffer): builds that name `level0` as their image copy nothing.
    nbytes: bytes readable from level0's first element (default: to the end
    of the tensor's storage); at least pitch * h + 32.  The handle keeps a
    reference to `level0`."""
    p, w, h, pitch, dev = _img_args(level0)
    if not dev:
        raise ValueError("level 0 must be a CUDA tensor")
    if nbytes is None:
        st = level0.untyped_storage()
        nbytes = st.data_ptr() + st.nbytes() - p
    hd = vp()
    _check(_lib.vt_pyramid_create_on(p, pitch, int(nbytes), w, h, levels, C.byref(hd)), "vt_pyramid_create_on")
    pyr = Pyramid(hd.value)
    pyr.level0 = level0
    return pyr


# ------------------------------------------------------------------ batched
class vt_frame_job(C.Structure):
    _fields_ = [("img", vp), ("pitch", i32), ("pyr", vp)]


class vt_track_task(C.Structure):
    _fields_ = [("prev", vp), ("cur", vp), ("pts_in", vp), ("n", i32), ("fb", i32), ("pts_out", vp),
                ("status", vp), ("err", vp), ("reason", vp), ("flops", vp), ("levels", i32), ("n_dev", vp)]


_sig("vt_batch_create", i32, [i32, i32, C.POINTER(vp)])
_sig("vt_batch_free", None, [vp])
_sig("vt_batch_config", i32, [vp, i32, i32, i32])
_sig("vt_batch_set", i32, [vp, C.POINTER(vt_frame_job), i32, i32, C.POINTER(vt_track_task), i32,
                           C.POINTER(vt_klt_params)])
_sig("vt_batch_run", i32, [vp, vp])
_sig("vt_batch_run_graph", i32, [vp, vp])
_sig("vt_batch_run_timed", i32, [vp, vp, vp, vp, vp, vp])
_sig("vt_batch_info", i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)])


def _event_handle(ev):
    """cudaEvent_t of a torch.cuda.Event (or an int handle, or None).  torch
    creates its events lazily, so a torch event must have been recorded once."""
    if ev is None or isinstance(ev, int):
        return ev
    h = ev.cuda_event
    if not h:
        raise ValueError("torch.cuda.Event has no CUDA event yet: record it once before passing it")
    return h


class Batch:
    """Owning handle of a vt_batch (batched persistent tracking)."""

    def __init__(self, max_frames: int, max_tasks: int):
        hd = vp()
        _check(_lib.vt_batch_create(max_frames, max_tasks, C.byref(hd)), "vt_batch_create")
        self.handle = hd.value
        self._keep = None

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)

    def free(self):
        if self.handle:
            _lib.vt_batch_free(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def vt_batch_create(max_frames: int, max_tasks: int) -> Batch:
    return Batch(max_frames, max_tasks)


def vt_batch_free(b: Batch) -> None:
    b.free()


def vt_batch_config(b: Batch, klt_warps_per_cta: int = 4, klt_ctas_per_sm: int = 0, pyr_ctas: int = 0) -> None:
    _check(_lib.vt_batch_config(b, klt_warps_per_cta, klt_ctas_per_sm, pyr_ctas), "vt_batch_config")


def frame_job(img, pyr: Pyramid) -> vt_frame_job:
    """Descriptor of one pyramid build from a 2-D uint8 device tensor, or a
    pinned host tensor (the pyramid kernel then reads it over the host link)."""
    p, w, h, pitch, dev = _img_args(img)
    if not dev and not (hasattr(img, "is_pinned") and img.is_pinned()):
        raise ValueError("batched frames must be device images or pinned host tensors")
    return vt_frame_job(p, pitch, pyr.handle)


def track_task(prev: Pyramid, cur: Pyramid, pts_in, pts_out, status, err=None, fb=True, reason=None,
               flops=None, levels=0, n_dev=None) -> vt_track_task:
    """n_dev: optional device int; only the first min(n, *n_dev) points are tracked."""
    return vt_track_task(prev.handle, cur.handle, _ptr(pts_in), int(pts_in.shape[0]), int(bool(fb)),
                         _ptr(pts_out), _ptr(status), _ptr(err), _ptr(reason), _ptr(flops), int(levels),
                         _ptr(n_dev))


def vt_batch_set(b: Batch, frames, tasks, params: KltParams, grad_type: int = VT_GRAD_S16) -> None:
    fa = (vt_frame_job * max(1, len(frames)))(*frames)
    ta = (vt_track_task * max(1, len(tasks)))(*tasks)
    prm = params.c()
    _check(_lib.vt_batch_set(b, fa, len(frames), grad_type, ta, len(tasks), C.byref(prm)), "vt_batch_set")


def vt_batch_run(b: Batch, stream=None) -> None:
    _check(_lib.vt_batch_run(b, _stream(stream)), "vt_batch_run")


def vt_batch_run_graph(b: Batch, stream=None) -> None:
    _check(_lib.vt_batch_run_graph(b, _stream(stream)), "vt_batch_run_graph")


def vt_batch_run_timed(b: Batch, stream=None, ev_pyr0=None, ev_pyr1=None, ev_klt0=None, ev_klt1=None) -> None:
    _check(_lib.vt_batch_run_timed(b, _stream(stream), _event_handle(ev_pyr0), _event_handle(ev_pyr1),
                                   _event_handle(ev_klt0), _event_handle(ev_klt1)), "vt_batch_run_timed")


_sig("vt_batch_run_levels_timed", i32, [vp, vp, C.POINTER(vp), i32])


def vt_batch_run_levels_timed(b: Batch, stream, events) -> None:
    """events: 4 + pyramid-launch CUDA events (see vt.h); None entries skipped."""
    arr = (vp * len(events))(*[_event_handle(e) for e in events])
    _check(_lib.vt_batch_run_levels_timed(b, _stream(stream), arr, len(events)), "vt_batch_run_levels_timed")


class vt_copy(C.Structure):
    _fields_ = [("dst", vp), ("src", vp), ("bytes", C.c_size_t)]


_sig("vt_copy_async", i32, [C.POINTER(vt_copy), i32, vp])


def vt_copy_async(copies, stream=None) -> None:
    """Issue copies given as (dst_ptr, src_ptr, bytes) tuples or a ctypes
    vt_copy array, in order, on ``stream``."""
    if isinstance(copies, C.Array):
        arr, n = copies, len(copies)
    else:
        lst = list(copies)
        arr = (vt_copy * max(1, len(lst)))(*[vt_copy(d, s_, b) for d, s_, b in lst])
        n = len(lst)
    _check(_lib.vt_copy_async(arr, n, _stream(stream)), "vt_copy_async")


def vt_batch_info(b: Batch):
    g, w, pg, nl = i32(), i32(), i32(), i32()
    _check(_lib.vt_batch_info(b, C.byref(g), C.byref(w), C.byref(pg), C.byref(nl)), "vt_batch_info")
    return dict(klt_grid=g.value, klt_warps=w.value, pyr_grid=pg.value, launches_per_run=nl.value)


_sig("vt_klt_track_tasks_noalloc", i32, [C.POINTER(vt_track_task), i32, C.POINTER(vt_klt_params), vp])


def vt_klt_track_tasks_noalloc(tasks, params: KltParams, stream=None) -> None:
    """Track every task of `tasks` (vt_track_task list) in one launch that
    allocates no device memory (see include/vt.h)."""
    ta = (vt_track_task * max(1, len(tasks)))(*tasks)
    prm = params.c()
    _check(_lib.vt_klt_track_tasks_noalloc(ta, len(tasks), C.byref(prm), _stream(stream)),
           "vt_klt_track_tasks_noalloc")


# ------------------------------------------------------------------ GFTT
class vt_gftt_params(C.Structure):
    _fields_ = [("max_corners", i32), ("quality", f32), ("min_dist", i32), ("nms_radius", i32),
                ("block_radius", i32), ("border", i32)]


_sig("vt_gftt_create", i32, [i32, i32, C.POINTER(vp)])
_sig("vt_gftt_free", None, [vp])
_sig("vt_gftt_detect", i32, [vp, vp, i32, C.POINTER(vt_gftt_params), vp, i32, vp, vp, vp, vp])


@dataclass
class GfttParams:
    max_corners: int = 150
    quality: float = 0.01
    min_dist: int = 10
    nms_radius: int = 4
    block_radius: int = 1
    border: int = 10

    def c(self) -> vt_gftt_params:
        return vt_gftt_params(self.max_corners, self.quality, self.min_dist, self.nms_radius, self.block_radius,
                              self.border)


class Gftt:
    """Owning handle of a vt_gftt detector workspace."""

    def __init__(self, max_w: int, max_h: int):
        hd = vp()
        _check(_lib.vt_gftt_create(max_w, max_h, C.byref(hd)), "vt_gftt_create")
        self.handle = hd.value

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)

    def free(self):
        if self.handle:
            _lib.vt_gftt_free(C.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def vt_gftt_create(max_w: int, max_h: int) -> Gftt:
    return Gftt(max_w, max_h)


class vt_gftt_job(C.Structure):
    _fields_ = [("pyr", vp), ("level", i32), ("mask_pts", vp), ("n_mask", i32), ("corners_out", vp),
                ("scores_out", vp), ("count_out", vp), ("max_corners", i32)]


_sig("vt_gftt_create_pixels", i32, [C.c_longlong, C.POINTER(vp)])
_sig("vt_gftt_detect_many", i32, [vp, C.POINTER(vt_gftt_job), i32, C.POINTER(vt_gftt_params), vp])


def vt_gftt_create_pixels(max_pixels: int) -> Gftt:
    g = Gftt.__new__(Gftt)
    hd = vp()
    _check(_lib.vt_gftt_create_pixels(int(max_pixels), C.byref(hd)), "vt_gftt_create_pixels")
    g.handle = hd.value
    return g


def gftt_job(pyr: Pyramid, level: int, corners_out, count_out, max_corners: int, scores_out=None,
             mask=None) -> vt_gftt_job:
    return vt_gftt_job(pyr.handle, level, _ptr(mask), 0 if mask is None else int(mask.shape[0]), _ptr(corners_out),
                       _ptr(scores_out), _ptr(count_out), int(max_corners))


def vt_gftt_detect_many(g: Gftt, jobs, params: GfttParams, stream=None) -> None:
    arr = (vt_gftt_job * max(1, len(jobs)))(*jobs)
    prm = params.c()
    _check(_lib.vt_gftt_detect_many(g, arr, len(jobs), C.byref(prm), _stream(stream)), "vt_gftt_detect_many")


def vt_gftt_free(g: Gftt) -> None:
    g.free()


def vt_gftt_detect(g: Gftt, pyr: Pyramid, level: int, params: GfttParams, corners_out, count_out, scores_out=None,
                   mask=None, stream=None) -> None:
    prm = params.c()
    n_mask = 0 if mask is None else int(mask.shape[0])
    _check(_lib.vt_gftt_detect(g, pyr, level, C.byref(prm), _ptr(mask), n_mask, _ptr(corners_out),
                               _ptr(scores_out), _ptr(count_out), _stream(stream)), "vt_gftt_detect")


# ------------------------------------------------------------------ stereo gate
class vt_stereo_rig(C.Structure):
    _fields_ = [("kl", C.c_double * 4), ("kr", C.c_double * 4), ("R", C.c_double * 9), ("t", C.c_double * 3)]


class vt_gate_params(C.Structure):
    _fields_ = [("min_disp", C.c_double), ("z_min", C.c_double), ("z_max", C.c_double),
                ("max_reproj", C.c_double)]


_sig("vt_stereo_gate", i32, [vp, vp, vp, i32, C.POINTER(vt_stereo_rig), C.POINTER(vt_gate_params), vp, vp, vp,
                             vp])

VT_LOST_DISP, VT_LOST_DEPTH, VT_LOST_REPROJ = 5, 6, 7


@dataclass
class StereoRig:
    """Pinhole intrinsics (fx, fy, cx, cy) of both cameras and the left-to-right
    extrinsics X_R = R X_L + t (R row-major, t in metres)."""
    kl: tuple
    kr: tuple
    R: tuple = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    t: tuple = (0.0, 0.0, 0.0)

    def c(self) -> vt_stereo_rig:
        import numpy as np

        def flat(v, n):
            a = np.asarray(v, np.float64).ravel()
            if a.size != n:
                raise ValueError(f"expected {n} values, got {a.size}")
            return (C.c_double * n)(*a.tolist())

        return vt_stereo_rig(flat(self.kl, 4), flat(self.kr, 4), flat(self.R, 9), flat(self.t, 3))


@dataclass
class GateParams:
    min_disp: float = 1.0
    z_min: float = 0.1
    z_max: float = 50.0
    max_reproj: float = 1.5

    def c(self) -> vt_gate_params:
        return vt_gate_params(self.min_disp, self.z_min, self.z_max, self.max_reproj)


def vt_stereo_gate(pts_l, pts_r, rig: StereoRig, params: GateParams, status_out, status_in=None, xyz_out=None,
                   reason_out=None, stream=None) -> None:
    n = int(pts_l.shape[0])
    r, p = rig.c(), params.c()
    _check(_lib.vt_stereo_gate(_ptr(pts_l), _ptr(pts_r), _ptr(status_in), n, C.byref(r), C.byref(p), _ptr(xyz_out),
                               _ptr(status_out), _ptr(reason_out), _stream(stream)), "vt_stereo_gate")


class vt_gate_task(C.Structure):
    _fields_ = [("pts_l", vp), ("pts_r", vp), ("status_in", vp), ("n", i32), ("rig", vt_stereo_rig), ("xyz", vp),
                ("status_out", vp), ("reason", vp)]


_sig("vt_batch_set_gates", i32, [vp, C.POINTER(vt_gate_task), i32, C.POINTER(vt_gate_params)])


def gate_task(pts_l, pts_r, rig: StereoRig, status_out, status_in=None, xyz=None, reason=None) -> vt_gate_task:
    return vt_gate_task(_ptr(pts_l), _ptr(pts_r), _ptr(status_in), int(pts_l.shape[0]), rig.c(), _ptr(xyz),
                        _ptr(status_out), _ptr(reason))


def vt_batch_set_gates(b: Batch, gates, params: GateParams) -> None:
    arr = (vt_gate_task * max(1, len(gates)))(*gates)
    prm = params.c()
    _check(_lib.vt_batch_set_gates(b, arr, len(gates), C.byref(prm)), "vt_batch_set_gates")


# ------------------------------------------------------------------ track bookkeeping
VT_POOL_MAX = 4096


class vt_track_pool(C.Structure):
    _fields_ = [("pts", vp), ("ids", vp), ("ages", vp), ("count", vp), ("next_id", vp), ("cap", i32)]


class vt_carry_job(C.Structure):
    _fields_ = [("pool", vt_track_pool), ("tracked", vp), ("status", vp), ("mask", vp)]


class vt_spawn_job(C.Structure):
    _fields_ = [("pool", vt_track_pool), ("corners", vp), ("n_corners", vp), ("accept", vp)]


_sig("vt_tracks_carry", i32, [C.POINTER(vt_carry_job), i32, f32, vp])
_sig("vt_tracks_spawn", i32, [C.POINTER(vt_spawn_job), i32, vp])


class TrackPool:
    """One stream's device-resident feature pool (positions, identities,
    ages, live count, next identity) of capacity `cap`."""

    def __init__(self, cap: int, device="cuda"):
        import torch

        self.cap = cap
        self.pts = torch.zeros((cap, 2), dtype=torch.float32, device=device)
        self.ids = torch.zeros(cap, dtype=torch.int32, device=device)
        self.ages = torch.zeros(cap, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.next_id = torch.zeros(1, dtype=torch.int32, device=device)

    def c(self) -> vt_track_pool:
        return vt_track_pool(_ptr(self.pts), _ptr(self.ids), _ptr(self.ages), _ptr(self.count), _ptr(self.next_id),
                             self.cap)


def carry_job(pool: TrackPool, tracked, status, mask=None) -> vt_carry_job:
    return vt_carry_job(pool.c(), _ptr(tracked), _ptr(status), _ptr(mask))


def spawn_job(pool: TrackPool, corners, n_corners, accept=None) -> vt_spawn_job:
    return vt_spawn_job(pool.c(), _ptr(corners), _ptr(n_corners), _ptr(accept))


def vt_tracks_carry(jobs, min_dist: float, stream=None) -> None:
    arr = (vt_carry_job * max(1, len(jobs)))(*jobs)
    _check(_lib.vt_tracks_carry(arr, len(jobs), min_dist, _stream(stream)), "vt_tracks_carry")


def vt_tracks_spawn(jobs, stream=None) -> None:
    arr = (vt_spawn_job * max(1, len(jobs)))(*jobs)
    _check(_lib.vt_tracks_spawn(arr, len(jobs), _stream(stream)), "vt_tracks_spawn")
