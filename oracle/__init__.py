"""CPU oracle of geometry-TSDF + asymmetric colour-volume integration.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The CUDA path in
``paper_1602_06645_gb300`` shares no code with it and never imports it.

``oracle.c`` is the plain per-voxel definition (Section IV.B, Eq. 5-7, 9 and
the inherited KinectFusion TSDF update; Eq. 8-10 as colour mode 1) in binary32
with a fixed operation order; ``adjoint.c`` is the binary64 photometric loss
and its analytic gradient (the calibration-refinement extension);
``raycast.c`` ray-casts the volumes (range, vertex, normal and colour maps);
``mesh.c`` extracts the zero level set as triangles and fills per-polygon
texture maps from the colour volume (Eq. 11-14); ``icp.c`` tracks the camera
(vertex / normal pyramid, projective point-to-plane ICP against the ray-cast
prediction, Section III).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("oracle.c", "adjoint.c", "raycast.c", "mesh.c", "icp.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

# -ffp-contract=off: no implicit fused multiply-adds; the operation order in the
# source is the definition.  No fast-math.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    srcs = [s for s in _SRCS if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("ng", ctypes.c_int32 * 3),
        ("nc", ctypes.c_int32 * 3),
        ("s_g", ctypes.c_float),
        ("s_c", ctypes.c_float),
        ("origin", ctypes.c_float * 3),
        ("mu", ctypes.c_float),
        ("max_weight", ctypes.c_int32),
        ("sigma", ctypes.c_float),
        ("band", ctypes.c_float),
        ("colour_mode", ctypes.c_int32),
        ("sample_mode", ctypes.c_int32),
        ("update_free_space", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
        ("zoff_g", ctypes.c_int32),
        ("zoff_c", ctypes.c_int32),
    ]


class AdjProblem(ctypes.Structure):
    _fields_ = [
        ("n_frames", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("images", ctypes.c_void_p), ("Rn", ctypes.c_void_p), ("tn", ctypes.c_void_p),
        ("offsets", ctypes.c_void_p), ("idx", ctypes.c_void_p),
        ("nc", ctypes.c_int32 * 3), ("s_c", ctypes.c_float), ("origin", ctypes.c_float * 3),
        ("T0", ctypes.c_double * 16),
    ]


class RcVolume(ctypes.Structure):
    _fields_ = [("ng", ctypes.c_int32 * 3), ("nc", ctypes.c_int32 * 3), ("s_g", ctypes.c_float),
                ("s_c", ctypes.c_float), ("origin", ctypes.c_float * 3), ("F", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("C", ctypes.c_void_p)]


class RcCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("Kinv", ctypes.c_float * 9),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("near_", ctypes.c_float),
                ("far_", ctypes.c_float), ("step_far", ctypes.c_float), ("step_near", ctypes.c_float),
                ("inv_sg", ctypes.c_float), ("inv_sc", ctypes.c_float)]


class MeshVolume(ctypes.Structure):
    _fields_ = [("ng", ctypes.c_int32 * 3), ("s_g", ctypes.c_float), ("origin", ctypes.c_float * 3),
                ("F", ctypes.c_void_p), ("W", ctypes.c_void_p)]


class ColourVolume(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int32 * 3), ("s_c", ctypes.c_float), ("origin", ctypes.c_float * 3),
                ("C", ctypes.c_void_p)]


class IcpLevel(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("Kl", ctypes.c_float * 9),
                ("V", ctypes.c_void_p), ("N", ctypes.c_void_p), ("PV", ctypes.c_void_p), ("PN", ctypes.c_void_p),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("Rp", ctypes.c_float * 9),
                ("tp", ctypes.c_float * 3), ("max_dist2", ctypes.c_float), ("min_cos", ctypes.c_float)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.orc_integrate.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp,
                                      ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
        lib.orc_integrate.restype = ctypes.c_int
        lib.orc_integrate_geometry.argtypes = [ctypes.POINTER(Params), vp, vp, vp, ctypes.c_int, ctypes.c_int,
                                               vp, vp]
        lib.orc_integrate_geometry.restype = ctypes.c_longlong
        lib.orc_frame_constants.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp, vp]
        lib.orc_params_size.restype = ctypes.c_int
        assert lib.orc_params_size() == ctypes.sizeof(Params)
        lib.orc_record_gates.argtypes = [ctypes.POINTER(Params), vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                         ctypes.c_longlong]
        lib.orc_record_gates.restype = ctypes.c_longlong
        lib.orc_adj_size.restype = ctypes.c_int
        assert lib.orc_adj_size() == ctypes.sizeof(AdjProblem)
        lib.orc_adj_voxels.argtypes = [ctypes.POINTER(AdjProblem), vp]
        lib.orc_adj_voxels.restype = ctypes.c_int64
        lib.orc_adj_cells.argtypes = [ctypes.POINTER(AdjProblem), vp, vp]
        lib.orc_adj_cells.restype = None
        lib.orc_adj_eval.argtypes = [ctypes.POINTER(AdjProblem), vp, vp, vp, ctypes.c_int64, vp, vp, vp, vp, vp,
                                     ctypes.c_int64, vp]
        lib.orc_hd_cells.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                     ctypes.c_int, vp, vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        lib.orc_hd_cells.restype = None
        lib.orc_adj_eval.restype = ctypes.c_double
        lib.orc_sparse_frame.argtypes = [ctypes.POINTER(Params), vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                         ctypes.c_int, vp, vp, vp, vp, ctypes.c_int64, vp, vp, vp, ctypes.c_int64,
                                         vp, vp, vp]
        lib.orc_sparse_frame.restype = ctypes.c_int
        lib.orc_raycast.argtypes = [ctypes.POINTER(RcVolume), ctypes.POINTER(RcCamera), vp, vp, vp, vp]
        lib.orc_raycast.restype = ctypes.c_longlong
        assert lib.orc_rc_sizes(0) == ctypes.sizeof(RcVolume) and lib.orc_rc_sizes(1) == ctypes.sizeof(RcCamera)
        lib.orc_mesh.argtypes = [ctypes.POINTER(MeshVolume), vp, ctypes.c_longlong]
        lib.orc_mesh.restype = ctypes.c_longlong
        lib.orc_icp_pyramid.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.orc_icp_level_K.argtypes = [vp, ctypes.c_int, vp]
        lib.orc_icp_maps.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        lib.orc_icp_system.argtypes = [ctypes.POINTER(IcpLevel), vp, vp, vp]
        lib.orc_icp_system.restype = ctypes.c_longlong
        lib.orc_icp_solve.argtypes = [vp, vp, vp]
        lib.orc_icp_solve.restype = ctypes.c_int
        lib.orc_icp_update.argtypes = [vp, vp]
        lib.orc_mesh_cubes.argtypes = [ctypes.POINTER(MeshVolume), vp, ctypes.c_longlong]
        lib.orc_mesh_cubes.restype = ctypes.c_longlong
        lib.orc_texture_sizes.argtypes = [vp, ctypes.c_longlong, ctypes.c_float, ctypes.c_int, vp]
        lib.orc_texture_sizes.restype = ctypes.c_longlong
        lib.orc_texture_fill.argtypes = [ctypes.POINTER(ColourVolume), vp, ctypes.c_longlong, vp, vp, vp]
        lib.orc_texture_fill.restype = None
        assert lib.orc_mesh_sizes(0) == ctypes.sizeof(MeshVolume) and lib.orc_mesh_sizes(1) == ctypes.sizeof(ColourVolume)
        _lib = lib
    return _lib


def _f32(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    assert a.shape == shape, (a.shape, shape)
    return a


def volume_geometry(dims_geo, voxel_size):
    """(s_g, s_c-independent) extent and default origin: the cube of
    dims_geo * voxel_size centred on the world origin."""
    return tuple(float(np.float32(-0.5 * float(n) * float(voxel_size))) for n in dims_geo)


def colour_voxel(dims_geo, dims_col, voxel_size):
    """Colour voxel size: the same physical extent split into dims_col voxels
    (Section IV.B: same size, more voxels), binary64 then rounded to binary32."""
    return float(np.float32(float(dims_geo[0]) * float(voxel_size) / float(dims_col[0])))


def slab_extent(dims_geo, dims_col, z0, z1):
    """Geometry and colour z ranges held by the z-slab [z0, z1) (geometry
    voxels) of a volume: the colour range covering the same slice of space,
    [z0 Nc / Ng, z1 Nc / Ng) (both must be whole voxels), and the geometry
    range widened by the one voxel on each side that the band gate's trilinear
    corners reach, clipped to the volume.  Returns (g0, g1, c0, c1)."""
    ng, nc = int(dims_geo[2]), int(dims_col[2])
    if not (0 <= z0 < z1 <= ng) or (z0 * nc) % ng or (z1 * nc) % ng:
        raise ValueError("slab [%d, %d) does not cut both volumes at whole voxels" % (z0, z1))
    return max(0, z0 - 1), min(ng, z1 + 1), z0 * nc // ng, z1 * nc // ng


def make_params(dims_geo, dims_col, voxel_size, mu, max_weight, sigma=0.020, band=None, colour_mode=0,
                sample_mode=0, update_free_space=1, origin=None, n_threads=1, slab=None):
    """orc_params for the two volumes (Section IV.B); slab = (z0, z1) makes
    them the z-slab [z0, z1) of the volume of dims_geo / dims_col (see
    slab_extent)."""
    p = Params()
    p.ng[:] = [int(v) for v in dims_geo]
    p.nc[:] = [int(v) for v in dims_col]
    if slab is not None:
        g0, g1, c0, c1 = slab_extent(dims_geo, dims_col, *slab)
        p.ng[2], p.nc[2] = g1 - g0, c1 - c0
        p.zoff_g, p.zoff_c = g0, c0
    p.s_g = float(voxel_size)
    p.s_c = colour_voxel(dims_geo, dims_col, voxel_size)
    o = volume_geometry(dims_geo, voxel_size) if origin is None else origin
    p.origin[:] = [float(v) for v in o]
    p.mu = float(mu)
    p.max_weight = int(max_weight)
    p.sigma = float(sigma)
    # default band: one colour voxel either side of the zero crossing, in
    # normalised TSDF units (binary32 quotient)
    p.band = float(np.float32(p.s_c) / np.float32(p.mu)) if band is None else float(band)
    p.colour_mode, p.sample_mode = int(colour_mode), int(sample_mode)
    p.update_free_space, p.n_threads = int(update_free_space), int(n_threads)
    return p


class Oracle:
    """Holds the two volumes (linear, x fastest) and integrates frames on the CPU."""

    def __init__(self, dims_geo, dims_col, voxel_size, mu, max_weight, sigma=0.020, band=None,
                 colour_mode=0, sample_mode=0, update_free_space=1, origin=None, n_threads=1, slab=None):
        self.lib = _load()
        self.p = make_params(dims_geo, dims_col, voxel_size, mu, max_weight, sigma, band, colour_mode, sample_mode,
                             update_free_space, origin, n_threads, slab)
        gx, gy, gz = self.p.ng
        cx, cy, cz = self.p.nc
        self.F = np.zeros((gz, gy, gx), dtype=np.float32)
        self.W = np.zeros((gz, gy, gx), dtype=np.uint8)
        self.C = np.zeros((cz, cy, cx), dtype=np.uint32)
        self.counts = np.zeros(2, dtype=np.int64)

    def integrate(self, depth, rgb, K_depth, K_rgb, T_world_depth, T_depth_rgb):
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        dh, dw = depth.shape
        ch, cw, _ = rgb.shape
        Kd, Kr = _f32(K_depth, (3, 3)), _f32(K_rgb, (3, 3))
        Twd, Tdr = _f32(T_world_depth, (4, 4)), _f32(T_depth_rgb, (4, 4))
        self.lib.orc_integrate(ctypes.byref(self.p), self.F.ctypes.data, self.W.ctypes.data, self.C.ctypes.data,
                               depth.ctypes.data, dw, dh, rgb.ctypes.data, cw, ch, Kd.ctypes.data, Kr.ctypes.data,
                               Twd.ctypes.data, Tdr.ctypes.data, self.counts.ctypes.data)
        return int(self.counts[0]), int(self.counts[1])

    def integrate_geometry(self, depth, K_depth, T_world_depth):
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        dh, dw = depth.shape
        Kd, Twd = _f32(K_depth, (3, 3)), _f32(T_world_depth, (4, 4))
        return int(self.lib.orc_integrate_geometry(ctypes.byref(self.p), self.F.ctypes.data, self.W.ctypes.data,
                                                   depth.ctypes.data, dw, dh, Kd.ctypes.data, Twd.ctypes.data))

    def frame_constants(self, K_depth, K_rgb, T_world_depth, T_depth_rgb):
        R = np.zeros(9, np.float32)
        t = np.zeros(3, np.float32)
        Kdi = np.zeros(9, np.float32)
        args = [_f32(K_depth, (3, 3)), _f32(K_rgb, (3, 3)), _f32(T_world_depth, (4, 4)), _f32(T_depth_rgb, (4, 4))]
        self.lib.orc_frame_constants(ctypes.byref(self.p), *[a.ctypes.data for a in args], R.ctypes.data,
                                     t.ctypes.data, Kdi.ctypes.data)
        return R.reshape(3, 3), t, Kdi.reshape(3, 3)

    def record_gates(self, depth, K_depth, T_world_depth):
        """Geometry update of one frame, then S_k: the colour voxels (linear
        indices, ascending) that pass the depth-side gates against the
        updated geometry."""
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        dh, dw = depth.shape
        Kd, Twd = _f32(K_depth, (3, 3)), _f32(T_world_depth, (4, 4))
        cap = int(np.prod(self.C.shape))
        out = np.empty(cap, dtype=np.uint32)
        n = self.lib.orc_record_gates(ctypes.byref(self.p), self.F.ctypes.data, self.W.ctypes.data, depth.ctypes.data,
                                      dw, dh, Kd.ctypes.data, Twd.ctypes.data, out.ctypes.data, cap)
        if n < 0:
            raise MemoryError("orc_record_gates: no memory for the gate flags")
        return out[:n].copy()

    @property
    def colour_rgb(self):
        """(Nz, Ny, Nx, 3) uint8 colours."""
        c = self.C
        return np.stack([(c >> (8 * k)) & 0xFF for k in range(3)], axis=-1).astype(np.uint8)

    @property
    def colour_weight(self):
        return (self.C >> 24).astype(np.uint8)


class SparseOracle:
    """The same frame updates as Oracle, applied only to sampled voxels: a set
    of geometry voxels and a set of colour voxels, each given by linear
    indices (x fastest).  The colour band gate reads its trilinear corners from
    the geometry samples, so the geometry set must hold every corner of every
    colour sample; corners it lacks are counted in `missing`."""

    def __init__(self, geo_index, col_index, dims_geo, dims_col, voxel_size, mu, max_weight, **kw):
        self.lib = _load()
        self.p = make_params(dims_geo, dims_col, voxel_size, mu, max_weight, **kw)
        self.geo_index = np.unique(np.asarray(geo_index, dtype=np.uint64))
        self.col_index = np.unique(np.asarray(col_index, dtype=np.uint64))
        self.F = np.zeros(len(self.geo_index), np.float32)
        self.W = np.zeros(len(self.geo_index), np.uint8)
        self.C = np.zeros(len(self.col_index), np.uint32)
        self.missing = np.zeros(1, np.int64)

    def integrate(self, depth, rgb, K_depth, K_rgb, T_world_depth, T_depth_rgb):
        depth = np.ascontiguousarray(depth, dtype=np.uint16)
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        dh, dw = depth.shape
        ch, cw, _ = rgb.shape
        Kd, Kr = _f32(K_depth, (3, 3)), _f32(K_rgb, (3, 3))
        Twd, Tdr = _f32(T_world_depth, (4, 4)), _f32(T_depth_rgb, (4, 4))
        self.lib.orc_sparse_frame(ctypes.byref(self.p), depth.ctypes.data, dw, dh, rgb.ctypes.data, cw, ch,
                                  Kd.ctypes.data, Kr.ctypes.data, Twd.ctypes.data, Tdr.ctypes.data,
                                  len(self.geo_index), self.geo_index.ctypes.data, self.F.ctypes.data,
                                  self.W.ctypes.data, len(self.col_index), self.col_index.ctypes.data,
                                  self.C.ctypes.data, self.missing.ctypes.data)
        return int(self.missing[0])


class Adjoint:
    """Binary64 photometric loss of the colour volume and its gradient with
    respect to theta = (fx, fy, cx, cy, rho, phi) (adjoint.c)."""

    def __init__(self, images, Rn, tn, S, dims_col, s_c, origin, T0):
        self.lib = _load()
        self.images = np.ascontiguousarray(images, dtype=np.float32)
        n, H, W, _ = self.images.shape
        self.Rn = np.ascontiguousarray(np.asarray(Rn, np.float32).reshape(n, 9))
        self.tn = np.ascontiguousarray(np.asarray(tn, np.float32).reshape(n, 3))
        self.offsets = np.zeros(n + 1, np.int64)
        self.offsets[1:] = np.cumsum([len(x) for x in S])
        self.idx = np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint32) for x in S]) if n else
                                        np.zeros(0, np.uint32))
        p = AdjProblem()
        p.n_frames, p.width, p.height = n, W, H
        p.images, p.Rn, p.tn = self.images.ctypes.data, self.Rn.ctypes.data, self.tn.ctypes.data
        p.offsets, p.idx = self.offsets.ctypes.data, self.idx.ctypes.data
        p.nc[:] = [int(v) for v in dims_col]
        p.s_c = float(s_c)
        p.origin[:] = [float(v) for v in origin]
        p.T0[:] = [float(v) for v in np.asarray(T0, np.float64).reshape(16)]
        self.p = p
        nv = self.lib.orc_adj_voxels(ctypes.byref(p), None)
        self.V = np.empty(nv, np.uint32)
        self.lib.orc_adj_voxels(ctypes.byref(p), self.V.ctypes.data)

    def cells(self, theta):
        th = np.ascontiguousarray(theta, np.float64)
        cells = np.empty(2 * len(self.idx), np.int32)
        self.lib.orc_adj_cells(ctypes.byref(self.p), th.ctypes.data, cells.ctypes.data)
        return cells

    def cells32(self, K4, T):
        """Cells of the binary32 camera K4 = (fx, fy, cx, cy), 4x4 T: the
        integer decision taken by the fusion oracle's own colour path (Eq. 5,
        Eq. 3, Eq. 4 projection and the bilinear footprint test of oracle.c),
        the same precision as the kernels."""
        fx, fy, cx, cy = [float(v) for v in np.asarray(K4, np.float32)]
        Kr = np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1]], np.float32).reshape(9)
        t = np.ascontiguousarray(np.asarray(T, np.float32).reshape(16))
        cells = np.empty(2 * len(self.idx), np.int32)
        n, H, W, _ = self.images.shape
        nc = (ctypes.c_int32 * 3)(*self.p.nc)
        org = (ctypes.c_float * 3)(*self.p.origin)
        self.lib.orc_hd_cells(nc, ctypes.c_float(self.p.s_c), org, n, self.Rn.ctypes.data, self.tn.ctypes.data,
                              self.offsets.ctypes.data, self.idx.ctypes.data, Kr.ctypes.data, t.ctypes.data, W, H,
                              cells.ctypes.data)
        return cells

    def eval(self, theta, cells, target=None, grad=False, query=None):
        th = np.ascontiguousarray(theta, np.float64)
        nV = len(self.V)
        C = np.empty((nV, 3), np.float64)
        n = np.empty(nV, np.int32)
        tg = None if target is None else np.ascontiguousarray(target, np.float64)
        g = np.empty(10, np.float64) if grad else None
        q = None if query is None else np.ascontiguousarray(query, np.int64).reshape(-1, 4)
        qg = None if q is None else np.empty(len(q), np.float64)
        loss = self.lib.orc_adj_eval(ctypes.byref(self.p), th.ctypes.data, np.ascontiguousarray(cells).ctypes.data,
                                     self.V.ctypes.data, nV, None if tg is None else tg.ctypes.data, C.ctypes.data,
                                     n.ctypes.data, None if g is None else g.ctypes.data,
                                     None if q is None else q.ctypes.data, 0 if q is None else len(q),
                                     None if qg is None else qg.ctypes.data)
        return dict(loss=loss, C=C, n=n, grad=g, qgrad=qg)


def raycast(F, W, C, s_g, s_c, origin, K, T_world_camera, size, near, far, step_far=None, step_near=None,
            mu=None):
    """Ray-cast linear volumes F, W (Nz, Ny, Nx) and packed colours C (or
    None) from a pinhole camera (raycast.c).  Steps default to half the
    truncation distance mu in truncated free space and half a geometry voxel
    elsewhere.  Returns dict(range (H, W), vertex (H, W, 3), normal (H, W, 3),
    rgbw (H, W), hits)."""
    lib = _load()
    F = np.ascontiguousarray(F, np.float32)
    W = np.ascontiguousarray(W, np.uint8)
    v = RcVolume()
    v.ng[:] = [F.shape[2], F.shape[1], F.shape[0]]
    v.s_g, v.s_c = float(s_g), float(s_c)
    v.origin[:] = [float(o) for o in origin]
    v.F, v.W = F.ctypes.data, W.ctypes.data
    if C is not None:
        C = np.ascontiguousarray(C, np.uint32)
        v.nc[:] = [C.shape[2], C.shape[1], C.shape[0]]
        v.C = C.ctypes.data
    c = RcCamera()
    c.width, c.height = int(size[0]), int(size[1])
    c.Kinv[:] = [float(x) for x in np.linalg.inv(np.asarray(K, np.float64)).astype(np.float32).reshape(9)]
    T = np.asarray(T_world_camera, np.float32)
    c.R[:] = [float(x) for x in T[:3, :3].reshape(9)]
    c.t[:] = [float(x) for x in T[:3, 3]]
    mu = 3.0 * s_g if mu is None else mu
    c.near_, c.far_ = float(near), float(far)
    c.step_far = float(np.float32(0.5 * mu)) if step_far is None else float(step_far)
    c.step_near = float(np.float32(0.5 * s_g)) if step_near is None else float(step_near)
    c.inv_sg = float(np.float32(1.0 / np.float64(np.float32(s_g))))
    c.inv_sc = float(np.float32(1.0 / np.float64(np.float32(s_c))))
    H, Wd = c.height, c.width
    out = dict(range=np.zeros((H, Wd), np.float32), vertex=np.zeros((H, Wd, 3), np.float32),
               normal=np.zeros((H, Wd, 3), np.float32), rgbw=np.zeros((H, Wd), np.uint32))
    out["hits"] = int(lib.orc_raycast(ctypes.byref(v), ctypes.byref(c), out["range"].ctypes.data,
                                      out["vertex"].ctypes.data, out["normal"].ctypes.data, out["rgbw"].ctypes.data))
    return out


def mesh(F, W, s_g, origin, method="cubes"):
    """Triangles (n, 3, 3) of the zero level set of linear volumes F, W
    (Nz, Ny, Nx) by marching cubes (method "cubes", the paper's Section IV.C)
    or marching tetrahedra ("tetrahedra"), in cell order (mesh.c)."""
    lib = _load()
    fn = {"cubes": lib.orc_mesh_cubes, "tetrahedra": lib.orc_mesh}[method]
    F = np.ascontiguousarray(F, np.float32)
    W = np.ascontiguousarray(W, np.uint8)
    v = MeshVolume()
    v.ng[:] = [F.shape[2], F.shape[1], F.shape[0]]
    v.s_g = float(s_g)
    v.origin[:] = [float(o) for o in origin]
    v.F, v.W = F.ctypes.data, W.ctypes.data
    n = int(fn(ctypes.byref(v), None, 0))
    out = np.zeros((n, 3, 3), np.float32)
    fn(ctypes.byref(v), out.ctypes.data, n)
    return out


def texture_maps(tris, C, s_c, origin, size_pixel, max_side=1024):
    """Per-triangle texture maps (Eq. 11-14, mesh.c): (wh (n, 2) int32,
    offsets (n + 1) int64, texels uint32 packed RGBA)."""
    lib = _load()
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    n = len(tris)
    wh = np.zeros((n, 2), np.int32)
    total = int(lib.orc_texture_sizes(tris.ctypes.data, n, float(size_pixel), int(max_side), wh.ctypes.data))
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(wh[:, 0].astype(np.int64) * wh[:, 1])
    assert off[-1] == total
    C = np.ascontiguousarray(C, np.uint32)
    cv = ColourVolume()
    cv.nc[:] = [C.shape[2], C.shape[1], C.shape[0]]
    cv.s_c = float(s_c)
    cv.origin[:] = [float(o) for o in origin]
    cv.C = C.ctypes.data
    texels = np.zeros(total, np.uint32)
    lib.orc_texture_fill(ctypes.byref(cv), tris.ctypes.data, n, wh.ctypes.data, off.ctypes.data, texels.ctypes.data)
    return wh, off, texels


# ------------------------------------------------------------------ ICP ----
ICP_ITERATIONS = (10, 5, 4)  # per pyramid level, finest first (KinectFusion's counts)
ICP_MAX_DIST = 0.1           # correspondence distance gate (m)
ICP_MIN_COS = float(np.float32(np.cos(np.radians(20.0))))  # normal-angle gate: 20 degrees


def icp_pyramid(depth, levels):
    """Depth pyramid in metres (icp.c): a list of float32 (H >> l, W >> l) maps."""
    lib = _load()
    depth = np.ascontiguousarray(depth, np.uint16)
    H, W = depth.shape
    sizes = [(H >> l, W >> l) for l in range(levels)]
    buf = np.zeros(sum(h * w for h, w in sizes), np.float32)
    lib.orc_icp_pyramid(depth.ctypes.data, W, H, levels, buf.ctypes.data)
    out, o = [], 0
    for h, w in sizes:
        out.append(buf[o:o + h * w].reshape(h, w).copy())
        o += h * w
    return out


def icp_level_K(K, l):
    lib = _load()
    K = np.ascontiguousarray(K, np.float32).reshape(9)
    out = np.zeros(9, np.float32)
    lib.orc_icp_level_K(K.ctypes.data, int(l), out.ctypes.data)
    return out.reshape(3, 3)


def icp_maps(d, Kl):
    """Vertex and normal maps (H, W, 3), camera frame, of a depth map in metres."""
    lib = _load()
    d = np.ascontiguousarray(d, np.float32)
    h, w = d.shape
    V = np.zeros((h, w, 3), np.float32)
    N = np.zeros((h, w, 3), np.float32)
    K = np.ascontiguousarray(Kl, np.float32).reshape(9)
    lib.orc_icp_maps(d.ctypes.data, w, h, K.ctypes.data, V.ctypes.data, N.ctypes.data)
    return V, N


def _world_to_camera(T):
    """(R^T, -R^T t) of a camera -> world pose: the transpose exactly, the
    translation in binary64 rounded once."""
    T = np.asarray(T, np.float32)
    R = T[:3, :3].astype(np.float64)
    return T[:3, :3].T.copy(), (-(R.T @ T[:3, 3].astype(np.float64))).astype(np.float32)


def icp_system(V, N, PV, PN, Kl, T_cur, T_prev, max_dist=ICP_MAX_DIST, min_cos=ICP_MIN_COS):
    """One level's normal equations at pose T_cur (icp.c): dict(A (6, 6),
    g (6,), err2, n)."""
    lib = _load()
    h, w = V.shape[:2]
    L = IcpLevel()
    L.w, L.h = w, h
    L.Kl[:] = [float(x) for x in np.asarray(Kl, np.float32).reshape(9)]
    arrs = [np.ascontiguousarray(a, np.float32) for a in (V, N, PV, PN)]
    L.V, L.N, L.PV, L.PN = [a.ctypes.data for a in arrs]
    Tc = np.asarray(T_cur, np.float64).astype(np.float32)
    L.R[:] = [float(x) for x in Tc[:3, :3].reshape(9)]
    L.t[:] = [float(x) for x in Tc[:3, 3]]
    Rp, tp = _world_to_camera(T_prev)
    L.Rp[:] = [float(x) for x in Rp.reshape(9)]
    L.tp[:] = [float(x) for x in tp]
    L.max_dist2 = float(np.float32(max_dist) * np.float32(max_dist))
    L.min_cos = float(min_cos)
    A = np.zeros(36)
    g = np.zeros(6)
    e = np.zeros(1)
    n = lib.orc_icp_system(ctypes.byref(L), A.ctypes.data, g.ctypes.data, e.ctypes.data)
    return dict(A=A.reshape(6, 6), g=g, err2=float(e[0]), n=int(n))


def icp_solve(A, g):
    lib = _load()
    A = np.ascontiguousarray(A, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    xi = np.zeros(6)
    ok = lib.orc_icp_solve(A.ctypes.data, g.ctypes.data, xi.ctypes.data)
    return xi if ok else None


def icp_update(xi, T):
    lib = _load()
    T = np.ascontiguousarray(T, np.float64).copy()
    xi = np.ascontiguousarray(xi, np.float64)
    lib.orc_icp_update(xi.ctypes.data, T.ctypes.data)
    return T


def track(F, W, s_g, origin, mu, depth, K, T_prev, T_init, levels=3, iterations=ICP_ITERATIONS,
          max_dist=ICP_MAX_DIST, min_cos=ICP_MIN_COS, near=0.1, far=4.0):
    """Camera tracking of one depth frame against the volumes (F, W): the
    depth pyramid and its vertex / normal maps; per level, coarsest first,
    the prediction ray-cast from T_prev with the level's intrinsics and the
    given number of Gauss-Newton steps T <- exp(xi^) T from T_init.  Returns
    (T (4, 4) binary64, list of per-iteration dict(level, n, err2, A, g))."""
    pyr = icp_pyramid(depth, levels)
    T = np.asarray(T_init, np.float64).copy()
    log = []
    for l in reversed(range(levels)):
        Kl = icp_level_K(K, l)
        h, w = pyr[l].shape
        pred = raycast(F, W, None, s_g, s_g, origin, Kl, T_prev, (w, h), near, far, mu=mu)
        V, N = icp_maps(pyr[l], Kl)
        for _ in range(iterations[l]):
            r = icp_system(V, N, pred["vertex"], pred["normal"], Kl, T, T_prev, max_dist, min_cos)
            r["level"] = l
            log.append(r)
            xi = icp_solve(r["A"], r["g"])
            if xi is not None:
                T = icp_update(xi, T)
    return T, log
