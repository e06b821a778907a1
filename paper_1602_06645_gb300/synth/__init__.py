"""Seeded synthetic RGB-D sequences (ray-traced analytic scenes).

Stands in for the paper's captured scans (Section V: a Kinect 640x480 depth
camera rigidly paired with an HD RGB camera, Section IV.A).  This module holds
no fusion arithmetic: it renders input images and camera poses only, and is the
one source of inputs shared by the CPU oracle and the CUDA path.

Every random draw comes from splitmix64 counters (seed, frame, pixel), so the
bytes of a frame depend only on its arguments.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

PRIM_PLANE, PRIM_BOX, PRIM_SPHERE = 0, 1, 2
ALB_CHECKER, ALB_NOISE, ALB_CONSTANT = 0, 1, 2


class Prim(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("albedo", ctypes.c_int32),
        ("c", ctypes.c_double * 3),
        ("e", ctypes.c_double * 3),
        ("col_a", ctypes.c_double * 3),
        ("col_b", ctypes.c_double * 3),
        ("scale", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_render_depth.argtypes = [ctypes.POINTER(Prim), ctypes.c_int, dp, dp, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p]
        lib.synth_render_rgb.argtypes = [ctypes.POINTER(Prim), ctypes.c_int, dp, dp, ctypes.c_int,
                                         ctypes.c_int, dp, ctypes.c_void_p]
        lib.synth_prim_size.restype = ctypes.c_int
        assert lib.synth_prim_size() == ctypes.sizeof(Prim)
        _lib = lib
    return _lib


# ---------------------------------------------------------------- RNG ----
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & _M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
    return x ^ (x >> 31)


class Counter:
    """Counter-based stream of uniforms/normals (splitmix64 of seed, index)."""

    def __init__(self, seed: int):
        self.key = splitmix64(seed & _M64)
        self.i = 0

    def u01(self) -> float:
        self.i += 1
        return ((splitmix64(self.key ^ self.i) >> 11) + 0.5) / 9007199254740992.0

    def normal(self) -> float:
        u1, u2 = self.u01(), self.u01()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.u01()


# -------------------------------------------------------------- scenes ---
@dataclass
class Scene:
    prims: list = field(default_factory=list)
    background: tuple = (24.0, 24.0, 32.0)

    def array(self):
        arr = (Prim * max(1, len(self.prims)))()
        for i, p in enumerate(self.prims):
            arr[i] = p
        return arr

    def add(self, kind, c, e, albedo=ALB_CHECKER, col_a=(200, 40, 40), col_b=(40, 40, 200),
            scale=0.02, seed=0):
        p = Prim()
        p.kind, p.albedo = kind, albedo
        p.c[:] = [float(v) for v in c]
        ee = list(e) + [0.0] * (3 - len(e))
        p.e[:] = [float(v) for v in ee]
        p.col_a[:] = [float(v) for v in col_a]
        p.col_b[:] = [float(v) for v in col_b]
        p.scale, p.seed = float(scale), int(seed) & _M64
        self.prims.append(p)
        return self


def scene_sphere_box_plane(seed: int = 1) -> Scene:
    """Sphere r=0.2 m resting on a box resting on a ground plane (1 m cube)."""
    s = Scene()
    s.add(PRIM_PLANE, (0, 0, -0.4), (0, 0, 0), ALB_CHECKER, (220, 220, 210), (60, 70, 80), 0.02)
    s.add(PRIM_BOX, (0, 0, -0.3), (0.15, 0.15, 0.1), ALB_CHECKER, (200, 50, 40), (250, 210, 60), 0.02)
    s.add(PRIM_SPHERE, (0, 0, 0), (0.2,), ALB_NOISE, (30, 120, 200), (240, 240, 250), 12.0, seed=seed)
    return s


def scene_random_primitives(seed: int, n: int = 20, extent: float = 2.0) -> Scene:
    """n random spheres/boxes (sizes 0.1-0.5 m) on a ground plane, cube of side `extent`."""
    rng = Counter(seed)
    half = extent / 2.0
    ground = -0.4 * extent
    s = Scene()
    s.add(PRIM_PLANE, (0, 0, ground), (0, 0, 0), ALB_CHECKER, (210, 210, 200), (70, 60, 50), 0.02)
    for i in range(n):
        size = rng.uniform(0.1, 0.5) * extent / 2.0
        x = rng.uniform(-0.7 * half, 0.7 * half)
        y = rng.uniform(-0.7 * half, 0.7 * half)
        ca = tuple(rng.uniform(20, 250) for _ in range(3))
        cb = tuple(rng.uniform(20, 250) for _ in range(3))
        if rng.u01() < 0.5:
            r = size / 2.0
            s.add(PRIM_SPHERE, (x, y, ground + r), (r,), ALB_NOISE, ca, cb, 10.0 / extent, seed=seed * 131 + i)
        else:
            e = (size / 2.0, rng.uniform(0.3, 1.0) * size / 2.0, rng.uniform(0.3, 1.0) * size / 2.0)
            s.add(PRIM_BOX, (x, y, ground + e[2]), e, ALB_CHECKER, ca, cb, 0.02)
    return s


def scene_plane_sphere(seed: int = 3) -> Scene:
    """Ground plane plus one sphere (1 m cube)."""
    s = Scene()
    s.add(PRIM_PLANE, (0, 0, -0.3), (0, 0, 0), ALB_CHECKER, (230, 230, 220), (40, 90, 60), 0.02)
    s.add(PRIM_SPHERE, (0, 0, -0.05), (0.25,), ALB_NOISE, (200, 60, 30), (250, 230, 120), 12.0, seed=seed)
    return s


# ---------------------------------------------------------------- rig ----
def intrinsics(fx, fy, cx, cy) -> np.ndarray:
    return np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1]], dtype=np.float32)


K_DEPTH = intrinsics(525.0, 525.0, 319.5, 239.5)
K_RGB_1080 = intrinsics(1050.0, 1050.0, 959.5, 539.5)
K_RGB_720 = intrinsics(700.0, 700.0, 639.5, 359.5)
DEPTH_SIZE = (640, 480)
RGB_1080 = (1920, 1080)
RGB_720 = (1280, 720)


def rot_axis_angle(axis, angle) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def rig_depth_to_rgb(baseline: float = 0.025, yaw_deg: float = 1.0) -> np.ndarray:
    """T_depth_rgb: maps depth-camera coordinates to RGB-camera coordinates
    (rotation about the camera y axis, translation along x)."""
    T = np.eye(4)
    T[:3, :3] = rot_axis_angle((0, 1, 0), math.radians(yaw_deg))
    T[:3, 3] = (-baseline, 0.0, 0.0)
    return T.astype(np.float32)


def look_at(pos, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """T_world_cam for a camera at `pos` looking at `target` (x right, y down, z forward)."""
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, dtype=np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, f, pos
    return T


def orbit_poses(n, radius, elev_deg, deg_per_frame, target=(0.0, 0.0, 0.0), elev_amp_deg=0.0,
                jitter_t=0.0, jitter_deg=0.0, seed=0, phase_deg=0.0) -> np.ndarray:
    """(n, 4, 4) float32 T_world_depth on an orbit around `target`.

    Elevation follows elev_deg + elev_amp_deg * sin(2 pi f / n).  Optional pose
    jitter: N(0, jitter_t) metres per axis and a rotation of N(0, jitter_deg)
    degrees about a random axis."""
    rng = Counter(seed ^ 0x5EED)
    out = np.zeros((n, 4, 4), dtype=np.float64)
    for f in range(n):
        az = math.radians(phase_deg + f * deg_per_frame)
        el = math.radians(elev_deg + elev_amp_deg * math.sin(2 * math.pi * f / max(n, 1)))
        pos = np.asarray(target) + radius * np.array([math.cos(el) * math.cos(az),
                                                      math.cos(el) * math.sin(az), math.sin(el)])
        T = look_at(pos, target)
        if jitter_t > 0 or jitter_deg > 0:
            dt = np.array([rng.normal() for _ in range(3)]) * jitter_t
            ax = np.array([rng.normal() for _ in range(3)])
            ang = math.radians(rng.normal() * jitter_deg)
            T[:3, :3] = T[:3, :3] @ rot_axis_angle(ax, ang)
            T[:3, 3] += dt
        out[f] = T
    return out.astype(np.float32)


# ------------------------------------------------------------- render ----
def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def render_depth(scene: Scene, K, T_world_cam, size=DEPTH_SIZE, seed=0, frame=0,
                 noise_coeff=1.5e-3, dropout=0.02, max_range=4.0) -> np.ndarray:
    """uint16 millimetre depth image (H, W) of `scene`; 0 marks invalid pixels."""
    lib = _load()
    W, H = size
    Kd = np.ascontiguousarray(np.asarray(K, dtype=np.float32).astype(np.float64))
    Td = np.ascontiguousarray(np.asarray(T_world_cam, dtype=np.float32).astype(np.float64))
    out = np.zeros((H, W), dtype=np.uint16)
    arr = scene.array()
    lib.synth_render_depth(arr, len(scene.prims), _dptr(Kd), _dptr(Td), W, H, int(seed) & _M64,
                           int(frame) & _M64, float(noise_coeff), float(dropout), float(max_range),
                           out.ctypes.data)
    return out


def render_rgb(scene: Scene, K, T_world_cam, size=RGB_1080) -> np.ndarray:
    """uint8 HWC RGB image (H, W, 3) of `scene` (unlit albedo)."""
    lib = _load()
    W, H = size
    Kd = np.ascontiguousarray(np.asarray(K, dtype=np.float32).astype(np.float64))
    Td = np.ascontiguousarray(np.asarray(T_world_cam, dtype=np.float64))
    bg = np.ascontiguousarray(np.asarray(scene.background, dtype=np.float64))
    out = np.zeros((H, W, 3), dtype=np.uint8)
    arr = scene.array()
    lib.synth_render_rgb(arr, len(scene.prims), _dptr(Kd), _dptr(Td), W, H, _dptr(bg), out.ctypes.data)
    return out


def rgb_pose(T_world_depth, T_depth_rgb) -> np.ndarray:
    """T_world_rgb = T_world_depth * inverse(T_depth_rgb), in float64."""
    return np.asarray(T_world_depth, np.float64) @ np.linalg.inv(np.asarray(T_depth_rgb, np.float64))


# ------------------------------------------------------------ sequences --
@dataclass
class Sequence:
    """A seeded RGB-D sequence plus the volume it is fused into."""
    name: str
    scene: Scene
    poses: np.ndarray            # (n, 4, 4) float32 T_world_depth
    K_depth: np.ndarray
    K_rgb: np.ndarray
    T_depth_rgb: np.ndarray
    depth_size: tuple
    rgb_size: tuple
    seed: int
    dims_geo: tuple
    dims_col: tuple
    voxel_size: float            # geometry voxel (m)
    mu: float
    max_weight: int
    noise_coeff: float = 1.5e-3
    dropout: float = 0.02

    @property
    def n_frames(self):
        return len(self.poses)

    def frame(self, f: int):
        """(depth uint16 (H,W), rgb uint8 (H,W,3)) of frame f."""
        T = self.poses[f]
        depth = render_depth(self.scene, self.K_depth, T, self.depth_size, self.seed, f,
                             self.noise_coeff, self.dropout)
        rgb = render_rgb(self.scene, self.K_rgb, rgb_pose(T, self.T_depth_rgb), self.rgb_size)
        return depth, rgb


def _vox(extent, n):
    return float(np.float32(extent / n))


def sequence_small(n_frames: int = 10, seed: int = 1, dims_geo=128, ratio=2) -> Sequence:
    """Small plain-fusion sequence: 128^3 geometry / 256^3 colour over a 1 m cube,
    sphere on a box on a ground plane, 0.8 m orbit at 36 deg/frame."""
    poses = orbit_poses(n_frames, 0.8, 25.0, 36.0, target=(0.0, 0.0, -0.1), seed=seed)
    vs = _vox(1.0, dims_geo)
    return Sequence("plain_small_128_256", scene_sphere_box_plane(seed), poses, K_DEPTH, K_RGB_1080,
                    rig_depth_to_rgb(), DEPTH_SIZE, RGB_1080, seed, (dims_geo,) * 3,
                    (dims_geo * ratio,) * 3, vs, float(np.float32(3 * vs)), 64)


def sequence_tracking(n_frames: int = 12, seed: int = 5, dims_geo=128, ratio=2, deg_per_frame=2.0) -> Sequence:
    """Camera-tracking sequence: the small scene (sphere on a box on a ground
    plane, 1 m cube) seen from a 0.8 m orbit moving 2 deg per frame with pose
    jitter of 2 mm / 0.2 deg, so consecutive poses differ by what a tracker
    must recover."""
    poses = orbit_poses(n_frames, 0.8, 25.0, deg_per_frame, target=(0.0, 0.0, -0.1), jitter_t=2e-3,
                        jitter_deg=0.2, seed=seed)
    vs = _vox(1.0, dims_geo)
    return Sequence("tracking_128", scene_sphere_box_plane(seed), poses, K_DEPTH, K_RGB_1080,
                    rig_depth_to_rgb(), DEPTH_SIZE, RGB_1080, seed, (dims_geo,) * 3,
                    (dims_geo * ratio,) * 3, vs, float(np.float32(3 * vs)), 64)


def sequence_scan(n_frames: int = 300, seed: int = 2, dims_geo=512, ratio=2, frame_stride=1) -> Sequence:
    """Scan-scale sequence: 512^3 geometry / 1024^3 colour over a 2 m cube, 20 random
    primitives on a ground plane, one orbit (1.2 deg/frame for 300 frames) of radius
    1.6 m, elevation 25 +- 10 deg, pose jitter 1 mm / 0.1 deg."""
    total = 300
    poses = orbit_poses(total, 1.6, 25.0, 360.0 / total, target=(0.0, 0.0, -0.3), elev_amp_deg=10.0,
                        jitter_t=1e-3, jitter_deg=0.1, seed=seed)
    idx = (np.arange(n_frames) * frame_stride) % total
    vs = _vox(2.0, dims_geo)
    return Sequence("plain_scan_512_1024", scene_random_primitives(seed, 20, 2.0), poses[idx], K_DEPTH,
                    K_RGB_1080, rig_depth_to_rgb(), DEPTH_SIZE, RGB_1080, seed, (dims_geo,) * 3,
                    (dims_geo * ratio,) * 3, vs, float(np.float32(3 * vs)), 64)


def sequence_sweep(dims_col: int, n_frames: int = 100, seed: int = 3, dims_geo: int = 256) -> Sequence:
    """Asymmetry sweep: 256^3 geometry, colour 256..1024^3 over a 1 m cube, plane +
    sphere, 3.6 deg/frame."""
    poses = orbit_poses(n_frames, 0.8, 30.0, 3.6, target=(0.0, 0.0, -0.1), seed=seed)
    vs = _vox(1.0, dims_geo)
    return Sequence("sweep_256_%d" % dims_col, scene_plane_sphere(seed), poses, K_DEPTH, K_RGB_1080,
                    rig_depth_to_rgb(), DEPTH_SIZE, RGB_1080, seed, (dims_geo,) * 3, (dims_col,) * 3,
                    vs, float(np.float32(3 * vs)), 64)


def batched_edges(n_scans: int = 64, seed0: int = 100):
    """Geometry edges n_i = 8 * round(exp(U(ln 64, ln 384)) / 8) for scans seed0.."""
    out = []
    for i in range(n_scans):
        r = Counter(seed0 + i)
        n = math.exp(r.uniform(math.log(64.0), math.log(384.0)))
        out.append(int(8 * round(n / 8.0)))
    return out


def sequence_batched_scan(i: int, n_frames: int = 30, seed0: int = 100, edge=None) -> Sequence:
    """Scan i of the batched workload: its own scene variant and orbit phase,
    colour volume 2x the geometry edge, 1 m cube, 720p RGB."""
    seed = seed0 + i
    n = edge if edge is not None else batched_edges(i + 1, seed0)[i]
    r = Counter(seed ^ 0xBA7C)
    scene = scene_random_primitives(seed, 3 + int(r.u01() * 4), 1.0)
    poses = orbit_poses(n_frames, 0.8, 25.0, 12.0, target=(0.0, 0.0, -0.15), seed=seed,
                        phase_deg=r.uniform(0, 360))
    vs = _vox(1.0, n)
    return Sequence("batched_%d_%d" % (i, n), scene, poses, K_DEPTH, K_RGB_720, rig_depth_to_rgb(),
                    DEPTH_SIZE, RGB_720, seed, (n,) * 3, (2 * n,) * 3, vs, float(np.float32(3 * vs)), 64)


def sequence_adjoint(n_frames: int = 20, seed: int = 4, dims_geo=256, ratio=2) -> Sequence:
    """Adjoint workload: 256^3 / 512^3 over a 1 m cube, 18 deg/frame."""
    poses = orbit_poses(n_frames, 0.8, 25.0, 18.0, target=(0.0, 0.0, -0.1), seed=seed)
    vs = _vox(1.0, dims_geo)
    return Sequence("adjoint_256_512", scene_sphere_box_plane(seed), poses, K_DEPTH, K_RGB_1080,
                    rig_depth_to_rgb(), DEPTH_SIZE, RGB_1080, seed, (dims_geo,) * 3,
                    (dims_geo * ratio,) * 3, vs, float(np.float32(3 * vs)), 64)
