"""Sample sets for parity checks at full size.

The voxels to compare are chosen from the synthetic inputs alone (depth maps
and poses), never from a result: colour voxels around back-projected depth
pixels, where the colour gates can pass; the geometry voxels around them,
which hold every trilinear corner the band gate reads; geometry voxels within
a truncation distance of the same points; and geometry voxels drawn uniformly
over the whole volume (mostly free space or never seen).
"""
import numpy as np


def _linear(ijk, dims):
    ijk = ijk.astype(np.int64)
    return (ijk[:, 2] * dims[1] + ijk[:, 1]) * dims[0] + ijk[:, 0]


def _inside(ijk, dims):
    return np.all((ijk >= 0) & (ijk < np.asarray(dims)), axis=1)


def surface_points(seq, frames, n_points, seed):
    """World points of n_points random valid depth pixels spread over `frames`."""
    rng = np.random.default_rng(seed)
    per = -(-n_points // len(frames))
    K = np.asarray(seq.K_depth, np.float64)
    out = []
    for f in frames:
        d, _ = seq.frame(f)
        v, u = np.nonzero(d)
        pick = rng.choice(len(u), size=min(per, len(u)), replace=False)
        u, v = u[pick].astype(np.float64), v[pick].astype(np.float64)
        z = d[v.astype(int), u.astype(int)].astype(np.float64) * 1e-3
        cam = np.stack([(u - K[0, 2]) / K[0, 0] * z, (v - K[1, 2]) / K[1, 1] * z, z, np.ones_like(z)], axis=1)
        out.append((np.asarray(seq.poses[f], np.float64) @ cam.T).T[:, :3])
    return np.concatenate(out)[:n_points]


def scan_samples(seq, frames, n_col, n_geo, seed=0):
    """(geometry linear indices, colour linear indices), ascending and unique."""
    rng = np.random.default_rng(seed)
    ng, nc = np.asarray(seq.dims_geo), np.asarray(seq.dims_col)
    s_g = float(seq.voxel_size)
    s_c = s_g * float(ng[0]) / float(nc[0])
    origin = -0.5 * ng * s_g
    # colour voxels: surface points jittered by up to two colour voxels
    P = surface_points(seq, frames, n_col, seed)
    P = P + rng.uniform(-2.0 * s_c, 2.0 * s_c, size=P.shape)
    c = np.floor((P - origin) / s_c).astype(np.int64)
    c = c[_inside(c, nc)]
    col = np.unique(_linear(c, nc))
    # their trilinear corners and one voxel more on each side
    cc = np.stack([col % nc[0], (col // nc[0]) % nc[1], col // (nc[0] * nc[1])], axis=1)
    g0 = np.floor((cc + 0.5) * s_c / s_g - 0.5).astype(np.int64)
    off = np.stack(np.meshgrid(*[np.arange(-1, 3)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    nb = (g0[:, None, :] + off[None, :, :]).reshape(-1, 3)
    nb = nb[_inside(nb, ng)]
    # geometry voxels near the surface (within the truncation distance) ...
    Q = surface_points(seq, frames, n_geo // 2, seed + 1)
    Q = Q + rng.uniform(-2.0 * float(seq.mu), 2.0 * float(seq.mu), size=Q.shape)
    g = np.floor((Q - origin) / s_g).astype(np.int64)
    g = g[_inside(g, ng)]
    # ... and anywhere in the volume
    u = rng.integers(0, ng, size=(n_geo - n_geo // 2, 3))
    geo = np.unique(np.concatenate([_linear(nb, ng), _linear(g, ng), _linear(u, ng)]))
    return geo.astype(np.uint64), col.astype(np.uint64)
