"""GB300-native geometry-TSDF + asymmetric colour-volume fusion.

Thin Python binding of the C ABI in ``include/tsdf.h`` (``libtsdf.so``): the
functions below carry the C names and only marshal arguments; every step of
fusion runs in the library's CUDA kernels.  PyTorch provides device memory
(through its caching allocator) and streams.

The library is loaded on first use; calling into it without the built
``libtsdf.so`` raises an error (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsdf.so")

TSDF_OK = 0
TSDF_ERR_INVALID_ARG = -1
TSDF_ERR_OOM = -2
TSDF_ERR_CUDA = -3
TSDF_ERR_TIMEOUT = -4
TSDF_ERR_DEVICE_FAULT = -5
TSDF_ERR_IO = -6
TSDF_COLOUR_COUNT, TSDF_COLOUR_PAPER_NORMAL = 0, 1
TSDF_SAMPLE_NEAREST, TSDF_SAMPLE_BILINEAR = 0, 1
TSDF_SCHEDULE_KERNELS, TSDF_SCHEDULE_FUSED = 0, 1

# symbols include/tsdf.h declares (checked by the tests)
EXPORTS = [
    "tsdf_params_default", "tsdf_create", "tsdf_create_ex", "tsdf_integrate", "tsdf_read", "tsdf_write",
    "tsdf_synchronize", "tsdf_save", "tsdf_load", "tsdf_destroy", "tsdf_set_stream", "tsdf_get_info",
    "tsdf_get_stats", "tsdf_stats_request", "tsdf_stats_collect", "tsdf_status_string", "tsdf_last_error", "tsdf_profile_enable", "tsdf_profile_read",
    "tsdf_integrate_geometry_static", "tsdf_adjoint_create", "tsdf_adjoint_record", "tsdf_adjoint_finalize",
    "tsdf_adjoint_voxels", "tsdf_adjoint_pairs", "tsdf_adjoint_forward", "tsdf_adjoint_backward",
    "tsdf_adjoint_destroy", "tsdf_batch_create", "tsdf_batch_integrate", "tsdf_batch_synchronize",
    "tsdf_batch_set_schedule", "tsdf_batch_get_schedule", "tsdf_batch_autotune", "tsdf_batch_inject_stall",
    "tsdf_batch_destroy", "tsdf_raycast", "tsdf_mesh", "tsdf_mesh_ex", "tsdf_texture_layout", "tsdf_texture_fill",
    "tsdf_profile_phases", "tsdf_track_params_default", "tsdf_track", "tsdf_set_frame_schedule",
    "tsdf_get_frame_schedule", "tsdf_fused_inject_stall", "tsdf_set_device_inputs_ready",
]
PHASES = ["upload", "depth_tiles", "bricks", "geometry", "colour_list", "colour_cells", "colour"]

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class tsdf_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class tsdf_params(ctypes.Structure):
    _fields_ = [
        ("origin", ctypes.c_float * 3),
        ("sigma", ctypes.c_float),
        ("band", ctypes.c_float),
        ("colour_mode", ctypes.c_int32),
        ("sample_mode", ctypes.c_int32),
        ("culling", ctypes.c_int32),
        ("update_free_space", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("allocator", tsdf_allocator),
        ("slab_z", ctypes.c_int32 * 2),
    ]


class tsdf_image_size(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class tsdf_info(ctypes.Structure):
    _fields_ = [
        ("dims_geo", ctypes.c_int32 * 3), ("dims_col", ctypes.c_int32 * 3),
        ("voxel_geo", ctypes.c_float), ("voxel_col", ctypes.c_float), ("origin", ctypes.c_float * 3),
        ("mu", ctypes.c_float), ("sigma", ctypes.c_float), ("band", ctypes.c_float),
        ("max_weight", ctypes.c_int32), ("colour_mode", ctypes.c_int32), ("sample_mode", ctypes.c_int32),
        ("culling", ctypes.c_int32), ("update_free_space", ctypes.c_int32),
        ("frames", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("slab_z", ctypes.c_int32 * 2), ("held_geo_z", ctypes.c_int32 * 2), ("held_col_z", ctypes.c_int32 * 2),
    ]


class tsdf_stats(ctypes.Structure):
    _fields_ = [
        ("geo_updated", ctypes.c_int64), ("col_updated", ctypes.c_int64), ("geo_bricks", ctypes.c_int64),
        ("col_bricks", ctypes.c_int64), ("visible_bricks", ctypes.c_int64), ("total_bricks", ctypes.c_int64),
        ("frames_counted", ctypes.c_int64), ("total_geo_updated", ctypes.c_int64),
        ("total_col_updated", ctypes.c_int64), ("total_geo_bricks", ctypes.c_int64),
        ("total_col_bricks", ctypes.c_int64), ("total_visible_bricks", ctypes.c_int64),
        ("total_col_active_bricks", ctypes.c_int64), ("total_cells", ctypes.c_int64),
        ("total_geo_changed_bricks", ctypes.c_int64),
    ]


class tsdf_profile_report(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("ms", ctypes.c_double * 7)]


class tsdf_frame(ctypes.Structure):
    _fields_ = [
        ("depth_mm", ctypes.c_void_p), ("dsz", tsdf_image_size), ("rgb_hwc", ctypes.c_void_p),
        ("csz", tsdf_image_size), ("K_depth", ctypes.POINTER(ctypes.c_float)),
        ("K_rgb", ctypes.POINTER(ctypes.c_float)), ("T_world_depth", ctypes.POINTER(ctypes.c_float)),
        ("T_depth_rgb", ctypes.POINTER(ctypes.c_float)),
    ]


class tsdf_track_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("iterations", ctypes.c_int32 * 3), ("max_distance", ctypes.c_float),
                ("min_normal_cos", ctypes.c_float), ("near_m", ctypes.c_float), ("far_m", ctypes.c_float)]


TRACK_MAX_STEPS = 32


class tsdf_track_report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("level", ctypes.c_int32 * TRACK_MAX_STEPS),
                ("solved", ctypes.c_int32 * TRACK_MAX_STEPS), ("correspondences", ctypes.c_int64 * TRACK_MAX_STEPS),
                ("err2", ctypes.c_double * TRACK_MAX_STEPS), ("A", (ctypes.c_double * 36) * TRACK_MAX_STEPS),
                ("g", (ctypes.c_double * 6) * TRACK_MAX_STEPS), ("T_before", (ctypes.c_double * 16) * TRACK_MAX_STEPS)]


class TsdfError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s (%d)%s" % (_status_text(status), status, (": " + msg) if msg else ""))


_lib = None


def _status_text(s):
    try:
        return load().tsdf_status_string(s).decode()
    except Exception:
        return "status"


def load():
    """Load libtsdf.so (built by ``__graft_entry__.build()``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtsdf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32p, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)
    H = ctypes.POINTER(ctypes.c_void_p)
    lib.tsdf_params_default.argtypes = [ctypes.POINTER(tsdf_params)]
    lib.tsdf_params_default.restype = None
    lib.tsdf_create.argtypes = [i32p, i32p, ctypes.c_float, ctypes.c_float, ctypes.c_int32, H]
    lib.tsdf_create_ex.argtypes = [i32p, i32p, ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                                   ctypes.POINTER(tsdf_params), H]
    lib.tsdf_integrate.argtypes = [vp, vp, tsdf_image_size, vp, tsdf_image_size, fp, fp, fp, fp]
    lib.tsdf_read.argtypes = [vp, vp, vp, vp]
    lib.tsdf_write.argtypes = [vp, vp, vp, vp]
    lib.tsdf_synchronize.argtypes = [vp]
    lib.tsdf_set_frame_schedule.argtypes = [vp, ctypes.c_int32]
    lib.tsdf_get_frame_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.tsdf_fused_inject_stall.argtypes = [vp]
    lib.tsdf_set_device_inputs_ready.argtypes = [vp, ctypes.c_int32]
    lib.tsdf_save.argtypes = [vp, ctypes.c_char_p]
    lib.tsdf_load.argtypes = [vp, ctypes.c_char_p]
    lib.tsdf_destroy.argtypes = [vp]
    lib.tsdf_destroy.restype = None
    lib.tsdf_set_stream.argtypes = [vp, vp]
    lib.tsdf_get_info.argtypes = [vp, ctypes.POINTER(tsdf_info)]
    lib.tsdf_get_stats.argtypes = [vp, ctypes.POINTER(tsdf_stats)]
    lib.tsdf_stats_request.argtypes = [vp, ctypes.c_int32]
    lib.tsdf_stats_collect.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(tsdf_stats)]
    lib.tsdf_status_string.argtypes = [ctypes.c_int]
    lib.tsdf_status_string.restype = ctypes.c_char_p
    lib.tsdf_last_error.argtypes = [vp]
    lib.tsdf_last_error.restype = ctypes.c_char_p
    lib.tsdf_integrate_geometry_static.argtypes = [i32p, ctypes.c_float, ctypes.c_float, ctypes.c_int32, fp, vp, vp,
                                                   vp, tsdf_image_size, fp, fp, vp]
    lib.tsdf_integrate_geometry_static.restype = ctypes.c_int
    lib.tsdf_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, H]
    lib.tsdf_batch_integrate.argtypes = [vp, ctypes.POINTER(tsdf_frame)]
    lib.tsdf_batch_synchronize.argtypes = [vp]
    lib.tsdf_batch_set_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    i32o = ctypes.POINTER(ctypes.c_int32)
    lib.tsdf_batch_get_schedule.argtypes = [vp, i32o, i32o, i32o, i32o]
    lib.tsdf_batch_autotune.argtypes = [vp, ctypes.POINTER(tsdf_frame), ctypes.c_int32, i32o, i32o,
                                        ctypes.POINTER(ctypes.c_float)]
    lib.tsdf_batch_inject_stall.argtypes = [vp]
    lib.tsdf_batch_destroy.argtypes = [vp]
    lib.tsdf_batch_destroy.restype = None
    for name in ("tsdf_batch_create", "tsdf_batch_integrate", "tsdf_batch_synchronize", "tsdf_batch_set_schedule",
                 "tsdf_batch_get_schedule", "tsdf_batch_autotune", "tsdf_batch_inject_stall"):
        getattr(lib, name).restype = ctypes.c_int
    lib.tsdf_adjoint_create.argtypes = [vp, ctypes.c_int32, ctypes.c_int64, H]
    lib.tsdf_adjoint_record.argtypes = [vp, vp, tsdf_image_size, fp, fp]
    lib.tsdf_adjoint_finalize.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.tsdf_adjoint_voxels.argtypes = [vp, vp]
    lib.tsdf_adjoint_pairs.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    lib.tsdf_adjoint_forward.argtypes = [vp, vp, tsdf_image_size, fp, fp, vp, vp]
    lib.tsdf_adjoint_backward.argtypes = [vp, vp, tsdf_image_size, fp, fp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.tsdf_adjoint_destroy.argtypes = [vp]
    lib.tsdf_adjoint_destroy.restype = None
    for name in ("tsdf_adjoint_create", "tsdf_adjoint_record", "tsdf_adjoint_finalize", "tsdf_adjoint_voxels",
                 "tsdf_adjoint_pairs", "tsdf_adjoint_forward", "tsdf_adjoint_backward"):
        getattr(lib, name).restype = ctypes.c_int
    lib.tsdf_raycast.argtypes = [vp, fp, fp, tsdf_image_size, ctypes.POINTER(tsdf_raycast_params), vp, vp, vp, vp]
    lib.tsdf_raycast.restype = ctypes.c_int
    lib.tsdf_mesh.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.tsdf_mesh_ex.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.tsdf_texture_layout.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, vp, vp]
    lib.tsdf_texture_fill.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
    for name in ("tsdf_mesh", "tsdf_mesh_ex", "tsdf_texture_layout", "tsdf_texture_fill"):
        getattr(lib, name).restype = ctypes.c_int
    lib.tsdf_track_params_default.argtypes = [ctypes.POINTER(tsdf_track_params)]
    lib.tsdf_track_params_default.restype = None
    lib.tsdf_track.argtypes = [vp, vp, tsdf_image_size, fp, fp, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(tsdf_track_params), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(tsdf_track_report)]
    lib.tsdf_track.restype = ctypes.c_int
    lib.tsdf_profile_enable.argtypes = [vp, ctypes.c_int32]
    lib.tsdf_profile_phases.argtypes = [vp, ctypes.c_uint32]
    lib.tsdf_profile_phases.restype = ctypes.c_int
    lib.tsdf_profile_read.argtypes = [vp, ctypes.POINTER(tsdf_profile_report)]
    for name in ("tsdf_create", "tsdf_create_ex", "tsdf_integrate", "tsdf_read", "tsdf_write", "tsdf_synchronize",
                 "tsdf_save", "tsdf_load", "tsdf_set_stream", "tsdf_get_info", "tsdf_get_stats",
                 "tsdf_stats_request", "tsdf_stats_collect", "tsdf_profile_enable", "tsdf_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class tsdf_raycast_params(ctypes.Structure):
    _fields_ = [("near_m", ctypes.c_float), ("far_m", ctypes.c_float), ("step_far", ctypes.c_float),
                ("step_near", ctypes.c_float)]


# ------------------------------------------------------------ marshalling --
def _check(status, handle=None):
    if status != TSDF_OK:
        msg = ""
        if handle:
            msg = load().tsdf_last_error(handle).decode()
        raise TsdfError(status, msg)


def _i32x3(v):
    return (ctypes.c_int32 * 3)(*[int(x) for x in v])


def _mat(a, n):
    """(binary32 copy of a matrix, a ctypes float array over it).  The array
    converts to the float* of the C signatures; built from the buffer it costs
    a third of a numpy ctypes pointer, which counts at one call per frame."""
    arr = np.array(a, dtype=np.float32, copy=True).reshape(-1)
    if arr.size != n:
        raise ValueError("expected %d values, got %d" % (n, arr.size))
    return arr, (ctypes.c_float * n).from_buffer(arr)


def _ptr(x, dtype, keep):
    """Host or device pointer of an image/volume argument (numpy array or torch tensor)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch tensor (CPU or CUDA)
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        keep.append(x)
        return ctypes.c_void_p(x.data_ptr())
    arr = np.ascontiguousarray(x, dtype=dtype)
    keep.append(arr)
    return ctypes.c_void_p(arr.ctypes.data)


def _hw(x):
    s = tuple(x.shape)
    return s[0], s[1]


def torch_allocator(device=None):
    """A tsdf_allocator drawing from PyTorch's CUDA caching allocator."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = tsdf_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


# ------------------------------------------------------------- C names ----
def tsdf_params_default():
    p = tsdf_params()
    load().tsdf_params_default(ctypes.byref(p))
    return p


def tsdf_create(dims_geo, dims_col, voxel_size, mu, max_weight):
    h = ctypes.c_void_p()
    _check(load().tsdf_create(_i32x3(dims_geo), _i32x3(dims_col), float(voxel_size), float(mu), int(max_weight),
                              ctypes.byref(h)))
    return h


def tsdf_create_ex(dims_geo, dims_col, voxel_size, mu, max_weight, params):
    h = ctypes.c_void_p()
    _check(load().tsdf_create_ex(_i32x3(dims_geo), _i32x3(dims_col), float(voxel_size), float(mu), int(max_weight),
                                 ctypes.byref(params), ctypes.byref(h)))
    return h


def tsdf_integrate(h, depth_mm, rgb_hwc, K_depth, K_rgb, T_world_depth, T_depth_rgb):
    keep = []
    dh, dw = _hw(depth_mm)
    ch, cw = _hw(rgb_hwc)
    dp = _ptr(depth_mm, np.uint16, keep)
    cp = _ptr(rgb_hwc, np.uint8, keep)
    mats = [_mat(K_depth, 9), _mat(K_rgb, 9), _mat(T_world_depth, 16), _mat(T_depth_rgb, 16)]
    _check(load().tsdf_integrate(h, dp, tsdf_image_size(dw, dh), cp, tsdf_image_size(cw, ch),
                                 *[m[1] for m in mats]), h)


def tsdf_read(h, tsdf=None, w_geo=None, rgbw=None):
    keep = []
    _check(load().tsdf_read(h, _ptr(tsdf, np.float32, keep), _ptr(w_geo, np.uint8, keep),
                            _ptr(rgbw, np.uint32, keep)), h)


def tsdf_write(h, tsdf=None, w_geo=None, rgbw=None):
    keep = []
    _check(load().tsdf_write(h, _ptr(tsdf, np.float32, keep), _ptr(w_geo, np.uint8, keep),
                             _ptr(rgbw, np.uint32, keep)), h)


def tsdf_raycast(h, K, T_world_camera, size, params=None, range_=None, vertex=None, normal=None, rgbw=None):
    keep = []
    mats = [_mat(K, 9), _mat(T_world_camera, 16)]
    _check(load().tsdf_raycast(h, mats[0][1], mats[1][1], tsdf_image_size(int(size[0]), int(size[1])),
                               ctypes.byref(params) if params is not None else None,
                               _ptr(range_, np.float32, keep), _ptr(vertex, np.float32, keep),
                               _ptr(normal, np.float32, keep), _ptr(rgbw, np.uint32, keep)), h)


TSDF_MESH_CUBES, TSDF_MESH_TETRAHEDRA = 0, 1


def tsdf_mesh(h, triangles=None, capacity=0):
    keep = []
    n = ctypes.c_int64()
    _check(load().tsdf_mesh(h, _ptr(triangles, np.float32, keep), int(capacity), ctypes.byref(n)), h)
    return n.value


def tsdf_mesh_ex(h, method, triangles=None, capacity=0):
    keep = []
    n = ctypes.c_int64()
    _check(load().tsdf_mesh_ex(h, int(method), _ptr(triangles, np.float32, keep), int(capacity), ctypes.byref(n)), h)
    return n.value


def tsdf_track_params_default():
    p = tsdf_track_params()
    load().tsdf_track_params_default(ctypes.byref(p))
    return p


def tsdf_track(h, depth_mm, K_depth, T_world_depth_prev, T_init, params=None, report=True):
    """Track a depth frame (tsdf_track): (T (4, 4) binary64, tsdf_track_report or None)."""
    keep = []
    dh, dw = _hw(depth_mm)
    Kd, Tp = _mat(K_depth, 9), _mat(T_world_depth_prev, 16)
    Ti = np.ascontiguousarray(np.asarray(T_init, np.float64).reshape(16))
    Tout = np.zeros(16, np.float64)
    rep = tsdf_track_report() if report else None
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().tsdf_track(h, _ptr(depth_mm, np.uint16, keep), tsdf_image_size(dw, dh), Kd[1], Tp[1],
                             Ti.ctypes.data_as(dp), None if params is None else ctypes.byref(params),
                             Tout.ctypes.data_as(dp), None if rep is None else ctypes.byref(rep)), h)
    return Tout.reshape(4, 4), rep


def tsdf_texture_layout(h, triangles, n, size_pixel, max_side, wh, offsets):
    keep = []
    _check(load().tsdf_texture_layout(h, _ptr(triangles, np.float32, keep), int(n), float(size_pixel),
                                      int(max_side), _ptr(wh, np.int32, keep), _ptr(offsets, np.int64, keep)), h)


def tsdf_texture_fill(h, triangles, n, wh, offsets, texels):
    keep = []
    _check(load().tsdf_texture_fill(h, _ptr(triangles, np.float32, keep), int(n), _ptr(wh, np.int32, keep),
                                    _ptr(offsets, np.int64, keep), _ptr(texels, np.uint32, keep)), h)


def tsdf_profile_phases(h, mask):
    _check(load().tsdf_profile_phases(h, int(mask)), h)


def tsdf_synchronize(h):
    _check(load().tsdf_synchronize(h), h)


def tsdf_set_frame_schedule(h, schedule):
    _check(load().tsdf_set_frame_schedule(h, int(schedule)), h)


def tsdf_get_frame_schedule(h):
    out = ctypes.c_int32()
    _check(load().tsdf_get_frame_schedule(h, ctypes.byref(out)), h)
    return out.value


def tsdf_fused_inject_stall(h):
    _check(load().tsdf_fused_inject_stall(h), h)


def tsdf_set_device_inputs_ready(h, ready):
    _check(load().tsdf_set_device_inputs_ready(h, int(ready)), h)


def tsdf_save(h, path):
    _check(load().tsdf_save(h, str(path).encode()), h)


def tsdf_load(h, path):
    _check(load().tsdf_load(h, str(path).encode()), h)


def tsdf_destroy(h):
    if h:
        load().tsdf_destroy(h)


def tsdf_set_stream(h, stream):
    _check(load().tsdf_set_stream(h, ctypes.c_void_p(int(stream or 0))), h)


def tsdf_get_info(h):
    o = tsdf_info()
    _check(load().tsdf_get_info(h, ctypes.byref(o)), h)
    return o


def tsdf_get_stats(h):
    o = tsdf_stats()
    _check(load().tsdf_get_stats(h, ctypes.byref(o)), h)
    return o


STATS_COPY_BYTES = 128  # TSDF_STATS_COPY_BYTES: bytes one counter read copies to the host


def tsdf_stats_request(h, slot):
    _check(load().tsdf_stats_request(h, int(slot)), h)


def tsdf_stats_collect(h, slot):
    o = tsdf_stats()
    _check(load().tsdf_stats_collect(h, int(slot), ctypes.byref(o)), h)
    return o


def tsdf_integrate_geometry_static(dims, voxel_size, mu, max_weight, origin, tsdf, w, depth_mm, K_depth,
                                   T_world_depth, stream=None):
    """Allocation-free geometry fusion into caller-owned device arrays (see
    include/tsdf.h): `tsdf` / `w` are CUDA tensors of dims[2] x dims[1] x
    dims[0] float32 / uint8, `depth_mm` a CUDA tensor of the depth image."""
    import torch

    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    for name, x, dts in (("tsdf", tsdf, (torch.float32,)), ("w", w, (torch.uint8,)),
                         ("depth_mm", depth_mm, (torch.int16, torch.uint16))):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype in dts and x.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA tensor of %s" % (name, " or ".join(map(str, dts))))
    if tsdf.numel() != n or w.numel() != n:
        raise ValueError("tsdf and w must hold dims[0] * dims[1] * dims[2] = %d elements" % n)
    if depth_mm.dim() != 2:
        raise ValueError("depth_mm must be a 2-D (height x width) tensor")
    keep = []
    dh, dw = _hw(depth_mm)
    org = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    Kd, Twd = _mat(K_depth, 9), _mat(T_world_depth, 16)
    _check(load().tsdf_integrate_geometry_static(_i32x3(dims), float(voxel_size), float(mu), int(max_weight),
                                                 org.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 _ptr(tsdf, np.float32, keep), _ptr(w, np.uint8, keep),
                                                 _ptr(depth_mm, np.uint16, keep), tsdf_image_size(dw, dh), Kd[1],
                                                 Twd[1], ctypes.c_void_p(int(stream or 0))))


def _frames(frames, keep):
    """tsdf_frame array from (depth, rgb, K_depth, K_rgb, T_world_depth, T_depth_rgb) tuples of
    CUDA tensors and host matrices."""
    arr = (tsdf_frame * len(frames))()
    for i, (d, c, Kd, Kr, Twd, Tdr) in enumerate(frames):
        dh, dw = _hw(d)
        ch, cw = _hw(c)
        mats = [_mat(Kd, 9), _mat(Kr, 9), _mat(Twd, 16), _mat(Tdr, 16)]
        keep.extend(mats)
        arr[i] = tsdf_frame(_ptr(d, np.uint16, keep), tsdf_image_size(dw, dh), _ptr(c, np.uint8, keep),
                            tsdf_image_size(cw, ch), *[m[1] for m in mats])
    return arr


def tsdf_batch_create(handles):
    b = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    _check(load().tsdf_batch_create(arr, len(handles), ctypes.byref(b)), handles[0])
    return b


def tsdf_batch_integrate(b, frames, err_handle=None):
    keep = []
    arr = _frames(frames, keep)
    _check(load().tsdf_batch_integrate(b, arr), err_handle)


def tsdf_batch_synchronize(b, err_handle=None):
    _check(load().tsdf_batch_synchronize(b), err_handle)


def tsdf_batch_set_schedule(b, blocks_per_sm, bricks_per_item=1, use_graph=True):
    _check(load().tsdf_batch_set_schedule(b, int(blocks_per_sm), int(bricks_per_item), int(bool(use_graph))))


def tsdf_batch_get_schedule(b):
    """(blocks per SM, max blocks per SM, bricks per item, use_graph)."""
    x, m, t, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().tsdf_batch_get_schedule(b, ctypes.byref(x), ctypes.byref(m), ctypes.byref(t), ctypes.byref(g)))
    return x.value, m.value, t.value, bool(g.value)


def tsdf_batch_autotune(b, frames, rounds=3):
    """Returns ((blocks per SM, bricks per item), median ms of every candidate,
    candidate (blocks - 1) * 4 + log2(bricks per item))."""
    keep = []
    arr = _frames(frames, keep)
    _, mx, _, _ = tsdf_batch_get_schedule(b)
    best, tile = ctypes.c_int32(), ctypes.c_int32()
    ms = (ctypes.c_float * (4 * mx))()
    _check(load().tsdf_batch_autotune(b, arr, int(rounds), ctypes.byref(best), ctypes.byref(tile), ms))
    return (best.value, tile.value), list(ms)


def tsdf_batch_inject_stall(b):
    _check(load().tsdf_batch_inject_stall(b))


def tsdf_batch_destroy(b):
    if b:
        load().tsdf_batch_destroy(b)


def tsdf_adjoint_create(h, max_frames, max_pairs):
    a = ctypes.c_void_p()
    _check(load().tsdf_adjoint_create(h, int(max_frames), int(max_pairs), ctypes.byref(a)), h)
    return a


def tsdf_adjoint_record(a, h, depth_mm, K_depth, T_world_depth):
    keep = []
    dh, dw = _hw(depth_mm)
    Kd, Twd = _mat(K_depth, 9), _mat(T_world_depth, 16)
    _check(load().tsdf_adjoint_record(a, _ptr(depth_mm, np.uint16, keep), tsdf_image_size(dw, dh), Kd[1], Twd[1]), h)


def tsdf_adjoint_finalize(a, h):
    n = ctypes.c_int64()
    _check(load().tsdf_adjoint_finalize(a, ctypes.byref(n)), h)
    return int(n.value)


def tsdf_adjoint_voxels(a, h, out):
    keep = []
    _check(load().tsdf_adjoint_voxels(a, _ptr(out, np.uint32, keep)), h)


def tsdf_adjoint_pairs(a, h, voxels=None, frames=None):
    keep = []
    n = ctypes.c_int64()
    _check(load().tsdf_adjoint_pairs(a, _ptr(voxels, np.uint32, keep), _ptr(frames, np.uint8, keep), ctypes.byref(n)), h)
    return int(n.value)


def tsdf_adjoint_forward(a, h, images, K4, T_depth_rgb, colours, counts):
    keep = []
    _, H, W, _ = tuple(images.shape)
    k4, T = _mat(K4, 4), _mat(T_depth_rgb, 16)
    _check(load().tsdf_adjoint_forward(a, _ptr(images, np.float32, keep), tsdf_image_size(W, H), k4[1], T[1],
                                       _ptr(colours, np.float32, keep), _ptr(counts, np.int32, keep)), h)


def tsdf_adjoint_backward(a, h, images, K4, T_depth_rgb, grad_colours, grad_images):
    keep = []
    _, H, W, _ = tuple(images.shape)
    k4, T = _mat(K4, 4), _mat(T_depth_rgb, 16)
    g = (ctypes.c_double * 10)()
    _check(load().tsdf_adjoint_backward(a, _ptr(images, np.float32, keep), tsdf_image_size(W, H), k4[1], T[1],
                                        _ptr(grad_colours, np.float32, keep), _ptr(grad_images, np.float32, keep), g), h)
    return np.array(list(g), dtype=np.float64)


def tsdf_adjoint_destroy(a):
    if a:
        load().tsdf_adjoint_destroy(a)


def tsdf_profile_enable(h, enable=True):
    _check(load().tsdf_profile_enable(h, int(bool(enable))), h)


def tsdf_profile_read(h):
    """{phase name: accumulated device ms} and the number of frames timed."""
    o = tsdf_profile_report()
    _check(load().tsdf_profile_read(h, ctypes.byref(o)), h)
    return {n: float(o.ms[i]) for i, n in enumerate(PHASES)}, int(o.frames)


def tsdf_status_string(s):
    return load().tsdf_status_string(int(s)).decode()


def tsdf_last_error(h):
    return load().tsdf_last_error(h).decode()


def slab_ranges(dims_geo, dims_col, n):
    """Split one volume's geometry z range into n contiguous z-slabs
    [z0, z1) for n devices, as equal as the cuts allow: every cut falls on a
    whole colour voxel and, where the slabs stay non-empty, on a multiple of
    the 8-voxel brick."""
    import math

    ngz, ncz = int(dims_geo[2]), int(dims_col[2])
    n = int(n)
    if n < 1 or n > ngz:
        raise ValueError("cannot cut %d geometry layers into %d slabs" % (ngz, n))
    unit = ngz // math.gcd(ngz, ncz)  # z0 * ncz / ngz is whole iff z0 is a multiple of unit
    for q in (unit * 8 // math.gcd(unit, 8), unit):
        cuts = [0] + [min(ngz, int(round(k * ngz / n / q)) * q) for k in range(1, n)] + [ngz]
        if all(a < b for a, b in zip(cuts, cuts[1:])):
            return list(zip(cuts, cuts[1:]))
    raise ValueError("no cut of %d layers into %d slabs falls on whole colour voxels" % (ngz, n))


def lpt_assign(costs, n):
    """Distribute independent scans over n devices by longest processing time
    first: scans in decreasing cost (ties by index) each go to the device with
    the least cost so far (ties to the lowest device).  Returns, per device,
    the indices of its scans in increasing order.  Deterministic, so every
    rank computes the same split without an exchange.  The slowest device's
    total is at most (4/3 - 1/(3n)) times the best possible (Graham's bound
    for the greedy rule)."""
    n = int(n)
    if n < 1:
        raise ValueError("need at least one device")
    costs = [float(c) for c in costs]
    if any(not (c >= 0.0) for c in costs):
        raise ValueError("costs must be non-negative numbers")
    load = [0.0] * n
    parts = [[] for _ in range(n)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        d = min(range(n), key=lambda r: (load[r], r))
        parts[d].append(i)
        load[d] += costs[i]
    return [sorted(p) for p in parts]


# ------------------------------------------------------------- Volume -----
class Volume:
    """A fusion handle with PyTorch-backed device memory on the current stream."""

    def __init__(self, dims_geo, dims_col, voxel_size, mu, max_weight, *, origin=None, sigma=0.020, band=None,
                 colour_mode=TSDF_COLOUR_COUNT, sample_mode=TSDF_SAMPLE_NEAREST, culling=True,
                 update_free_space=True, stream=None, torch_memory=True, slab=None, schedule=None,
                 device_inputs_ready=False):
        """slab = (z0, z1): hold the z-slab [z0, z1) of the volume (see
        tsdf_create_ex); dims_geo / dims_col are the whole volume's.
        schedule: TSDF_SCHEDULE_KERNELS or TSDF_SCHEDULE_FUSED (see
        tsdf_set_frame_schedule); None keeps the library's default.
        device_inputs_ready: see tsdf_set_device_inputs_ready."""
        import torch

        self.dims_geo = tuple(int(v) for v in dims_geo)
        self.dims_col = tuple(int(v) for v in dims_col)
        p = tsdf_params_default()
        if slab is not None:
            p.slab_z[:] = [int(slab[0]), int(slab[1])]
        if origin is not None:
            p.origin[:] = [float(v) for v in origin]
        p.sigma = float(sigma)
        if band is not None:
            p.band = float(band)
        p.colour_mode, p.sample_mode = int(colour_mode), int(sample_mode)
        p.culling, p.update_free_space = int(bool(culling)), int(bool(update_free_space))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        p.stream = ctypes.c_void_p(int(stream))
        self.stream = int(stream)
        if torch_memory:
            self._alloc = torch_allocator()
            p.allocator = self._alloc
        self.h = tsdf_create_ex(self.dims_geo, self.dims_col, voxel_size, mu, max_weight, p)
        info = tsdf_get_info(self.h)
        self.slab = (info.slab_z[0], info.slab_z[1])
        self.held_geo_z = (info.held_geo_z[0], info.held_geo_z[1])
        self.held_col_z = (info.held_col_z[0], info.held_col_z[1])
        if schedule is not None:
            tsdf_set_frame_schedule(self.h, schedule)
        if device_inputs_ready:
            tsdf_set_device_inputs_ready(self.h, 1)

    @property
    def schedule(self):
        return tsdf_get_frame_schedule(self.h)

    @schedule.setter
    def schedule(self, value):
        tsdf_set_frame_schedule(self.h, value)

    def _held_shapes(self):
        gx, gy, _ = self.dims_geo
        cx, cy, _ = self.dims_col
        return ((self.held_geo_z[1] - self.held_geo_z[0], gy, gx), (self.held_col_z[1] - self.held_col_z[0], cy, cx))

    def integrate(self, depth_mm, rgb_hwc, K_depth, K_rgb, T_world_depth, T_depth_rgb):
        tsdf_integrate(self.h, depth_mm, rgb_hwc, K_depth, K_rgb, T_world_depth, T_depth_rgb)

    def read(self):
        """(F, w, rgbw) as numpy arrays shaped (Nz, Ny, Nx), linear x-fastest
        (for a z-slab handle: the held z ranges, see read_slab)."""
        sg, sc = self._held_shapes()
        F = np.empty(sg, np.float32)
        W = np.empty(sg, np.uint8)
        C = np.empty(sc, np.uint32)
        tsdf_read(self.h, F, W, C)
        return F, W, C

    def read_slab(self):
        """The slab's own part (F and w of geometry z [z0, z1), the colour
        held): concatenated over the slabs of a volume in z order, these are
        the whole volume's arrays."""
        F, W, C = self.read()
        a = self.slab[0] - self.held_geo_z[0]
        b = a + self.slab[1] - self.slab[0]
        return F[a:b], W[a:b], C

    def read_torch(self, device="cuda"):
        """(F, w, rgbw) as device tensors (rgbw as int32 holding the packed bits)."""
        import torch

        sg, sc = self._held_shapes()
        F = torch.empty(sg, dtype=torch.float32, device=device)
        W = torch.empty(sg, dtype=torch.uint8, device=device)
        C = torch.empty(sc, dtype=torch.int32, device=device)
        tsdf_read(self.h, F, W, C)
        return F, W, C

    def raycast(self, K, T_world_camera, size, near=0.1, far=4.0, step_far=0.0, step_near=0.0, device=None):
        """Ray-cast the volumes from a camera (tsdf_raycast): dict of range
        (H, W), vertex and normal (H, W, 3) and rgbw (H, W, packed), as numpy
        arrays, or as device tensors when device is given."""
        w, h = int(size[0]), int(size[1])
        p = tsdf_raycast_params(float(near), float(far), float(step_far), float(step_near))
        if device is None:
            out = dict(range=np.empty((h, w), np.float32), vertex=np.empty((h, w, 3), np.float32),
                       normal=np.empty((h, w, 3), np.float32), rgbw=np.empty((h, w), np.uint32))
        else:
            import torch
            out = dict(range=torch.empty((h, w), dtype=torch.float32, device=device),
                       vertex=torch.empty((h, w, 3), dtype=torch.float32, device=device),
                       normal=torch.empty((h, w, 3), dtype=torch.float32, device=device),
                       rgbw=torch.empty((h, w), dtype=torch.int32, device=device))
        tsdf_raycast(self.h, K, T_world_camera, (w, h), p, out["range"], out["vertex"], out["normal"], out["rgbw"])
        return out

    def mesh(self, capacity=None, device=None, method="cubes"):
        """Triangles (n, 3, 3) of the TSDF zero level set (tsdf_mesh_ex: marching
        "cubes" or "tetrahedra"), in no fixed order; numpy, or a device tensor
        when device is given."""
        m = {"cubes": TSDF_MESH_CUBES, "tetrahedra": TSDF_MESH_TETRAHEDRA}[method]
        if capacity is None:
            capacity = tsdf_mesh_ex(self.h, m, None, 0)
        if device is None:
            out = np.empty((int(capacity), 3, 3), np.float32)
        else:
            import torch
            out = torch.empty((int(capacity), 3, 3), dtype=torch.float32, device=device)
        n = tsdf_mesh_ex(self.h, m, out if capacity else None, capacity)
        return out[:min(n, int(capacity))]

    def texture_maps(self, triangles, size_pixel, max_side=1024):
        """Per-triangle texture maps (tsdf_texture_layout + tsdf_texture_fill):
        (wh (n, 2), offsets (n + 1), texels) as numpy arrays, or as device
        tensors when triangles is a device tensor."""
        n = len(triangles)
        if hasattr(triangles, "is_cuda") and triangles.is_cuda:
            import torch
            dev = triangles.device
            tri = triangles.reshape(n, 9).contiguous()
            wh = torch.empty((n, 2), dtype=torch.int32, device=dev)
            off = torch.empty(n + 1, dtype=torch.int64, device=dev)
            tsdf_texture_layout(self.h, tri, n, size_pixel, max_side, wh, off)
            tex = torch.empty(int(off[n].item()), dtype=torch.int32, device=dev)
        else:
            tri = np.ascontiguousarray(triangles, np.float32).reshape(n, 9)
            wh = np.empty((n, 2), np.int32)
            off = np.empty(n + 1, np.int64)
            tsdf_texture_layout(self.h, tri, n, size_pixel, max_side, wh, off)
            tex = np.empty(int(off[n]), np.uint32)
        tsdf_texture_fill(self.h, tri, n, wh, off, tex)
        return wh, off, tex

    def write(self, F=None, W=None, C=None):
        tsdf_write(self.h, F, W, C)

    def synchronize(self):
        tsdf_synchronize(self.h)

    def stats(self):
        return tsdf_get_stats(self.h)

    def stats_request(self, slot):
        """Queue a copy of the counters into slot 0 or 1 without waiting."""
        tsdf_stats_request(self.h, slot)

    def stats_collect(self, slot):
        """Wait for slot's last copy and return it as stats() would have."""
        return tsdf_stats_collect(self.h, slot)

    def info(self):
        return tsdf_get_info(self.h)

    def profile_phases(self, phases):
        """Time only the named phases (see PHASES) from now on."""
        mask = 0
        for name in phases:
            mask |= 1 << PHASES.index(name)
        tsdf_profile_phases(self.h, mask)

    def profile(self, enable=True):
        tsdf_profile_enable(self.h, enable)

    def profile_read(self):
        return tsdf_profile_read(self.h)

    def save(self, path):
        tsdf_save(self.h, path)

    def load(self, path):
        tsdf_load(self.h, path)

    def close(self):
        if getattr(self, "h", None):
            tsdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many volumes fused together: one persistent, graph-captured launch per step."""

    def __init__(self, volumes):
        self.volumes = list(volumes)
        self.b = tsdf_batch_create([v.h for v in self.volumes])

    def integrate(self, frames):
        """frames[i] = (depth, rgb, K_depth, K_rgb, T_world_depth, T_depth_rgb) for volume i; images on the GPU."""
        tsdf_batch_integrate(self.b, frames, self.volumes[0].h)

    def synchronize(self):
        tsdf_batch_synchronize(self.b, self.volumes[0].h)

    def set_schedule(self, blocks_per_sm, use_graph=True, bricks_per_item=1):
        tsdf_batch_set_schedule(self.b, blocks_per_sm, bricks_per_item, use_graph)

    def schedule(self):
        return tsdf_batch_get_schedule(self.b)

    def autotune(self, frames, rounds=3):
        return tsdf_batch_autotune(self.b, frames, rounds)

    def close(self):
        if getattr(self, "b", None):
            tsdf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
