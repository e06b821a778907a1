"""Photometric colour loss of the fused colour volume, differentiable with
respect to the HD images, the HD intrinsics (Eq. 4) and the depth-to-HD
extrinsic (Eq. 3): a torch.autograd.Function over the library's hand-written
forward and adjoint kernels (tsdf_adjoint_* in include/tsdf.h).

Typical use (calibration refinement): record the depth sequence once, then
iterate  C = fuse(images, K, xi); loss = ((C - target)^2).sum();
loss.backward(); update K and T <- exp(-lr * grad_xi^) T, keeping xi = 0.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (Volume, tsdf_adjoint_backward, tsdf_adjoint_create, tsdf_adjoint_destroy, tsdf_adjoint_finalize,
               tsdf_adjoint_forward, tsdf_adjoint_pairs, tsdf_adjoint_record, tsdf_adjoint_voxels)


def se3_exp(xi) -> np.ndarray:
    """4x4 exp(xi^) for xi = (rho, phi), translation first (binary64)."""
    xi = np.asarray(xi, np.float64).reshape(6)
    rho, phi = xi[:3], xi[3:]
    a = float(np.linalg.norm(phi))
    W = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if a < 1e-4:
        A, B, C = 1 - a * a / 6, 0.5 - a * a / 24, 1.0 / 6 - a * a / 120
    else:
        A, B, C = math.sin(a) / a, (1 - math.cos(a)) / a ** 2, (a - math.sin(a)) / a ** 3
    T = np.eye(4)
    T[:3, :3] = np.eye(3) + A * W + B * W @ W
    T[:3, 3] = (np.eye(3) + B * W + C * W @ W) @ rho
    return T


class Adjoint:
    """Gate recording over a depth sequence plus forward / backward passes.

    The geometry volume lives in `volume` (a Volume); colours are not fused
    here, only the depth-side gate sets S_k are recorded."""

    def __init__(self, volume: Volume, max_frames: int, max_pairs: int = 1 << 24):
        self.vol = volume
        self.a = tsdf_adjoint_create(volume.h, max_frames, max_pairs)
        self.n_frames = 0
        self.n_voxels = None

    def record(self, depth_mm, K_depth, T_world_depth):
        tsdf_adjoint_record(self.a, self.vol.h, depth_mm, K_depth, T_world_depth)
        self.n_frames += 1

    def finalize(self):
        self.n_voxels = tsdf_adjoint_finalize(self.a, self.vol.h)
        self.voxels = torch.empty(self.n_voxels, dtype=torch.int32, device="cuda")
        if self.n_voxels:
            tsdf_adjoint_voxels(self.a, self.vol.h, self.voxels)
        return self.n_voxels

    def pairs(self):
        n = tsdf_adjoint_pairs(self.a, self.vol.h)
        vox = np.empty(n, np.uint32)
        fr = np.empty(n, np.uint8)
        if n:
            tsdf_adjoint_pairs(self.a, self.vol.h, vox, fr)
        return vox, fr

    def forward(self, images, K4, T_depth_rgb):
        C = torch.empty((self.n_voxels, 3), dtype=torch.float32, device="cuda")
        n = torch.empty(self.n_voxels, dtype=torch.int32, device="cuda")
        if self.n_voxels:
            tsdf_adjoint_forward(self.a, self.vol.h, images, K4, T_depth_rgb, C, n)
        return C, n

    def backward(self, images, K4, T_depth_rgb, grad_C, grad_images):
        if not self.n_voxels:
            return np.zeros(10)
        return tsdf_adjoint_backward(self.a, self.vol.h, images, K4, T_depth_rgb, grad_C, grad_images)

    def close(self):
        if getattr(self, "a", None):
            tsdf_adjoint_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ColourFusionFn(torch.autograd.Function):
    """C = fuse(images, K4, xi): the mean bilinear HD colour of every recorded
    colour voxel at the camera K4 = (fx, fy, cx, cy), T = exp(xi^) T0.

    Gradients: images (float32, like images), K4 (4), and xi (6) as the
    derivative with respect to a left perturbation of T(xi) = exp(xi^) T0.
    That is the gradient with respect to xi only at xi = 0, so xi must be zero:
    to move the camera, fold a step into T0 (T0 <- exp(step^) T0) and evaluate
    again at xi = 0.  A non-zero xi raises ValueError."""

    @staticmethod
    def forward(ctx, images, K4, xi, adj: Adjoint, T0):
        xi_np = xi.detach().cpu().numpy()
        if np.any(xi_np != 0):
            raise ValueError("ColourFusionFn is linearised at xi = 0: fold xi into T0 (T0 <- exp(xi^) T0) "
                             "and pass xi = 0")
        T = np.asarray(T0, np.float64).astype(np.float32)
        k4 = K4.detach().cpu().numpy().astype(np.float32)
        C, n = adj.forward(images.detach().contiguous(), k4, T)
        ctx.adj, ctx.T, ctx.k4 = adj, T, k4
        ctx.k_like = (K4.device, K4.dtype)
        ctx.xi_like = (xi.device, xi.dtype)
        ctx.save_for_backward(images)
        ctx.mark_non_differentiable(n)
        return C, n

    @staticmethod
    def backward(ctx, grad_C, grad_n):
        (images,) = ctx.saved_tensors
        gI = torch.zeros_like(images)
        g = ctx.adj.backward(images.contiguous(), ctx.k4, ctx.T, grad_C.contiguous().float(), gI)
        gK = torch.tensor(g[:4], dtype=ctx.k_like[1], device=ctx.k_like[0])
        gxi = torch.tensor(g[4:], dtype=ctx.xi_like[1], device=ctx.xi_like[0])
        return gI, gK, gxi, None, None


def fuse_colours(images, K4, xi, adj: Adjoint, T0):
    """Differentiable fused colours (n_voxels x 3) and sample counts."""
    return ColourFusionFn.apply(images, K4, xi, adj, T0)
