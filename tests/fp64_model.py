"""Independent binary64 evaluation of the fusion step, vectorised with numpy.

Used by the oracle pins only.  It follows Section IV.B (Eq. 5-7, 9), the
inherited KinectFusion TSDF update and the trilinear band gate, written from
the equations rather than from the oracle's source: positions, projections and
gates are evaluated in binary64 and every decision that lies within a small
margin of its threshold is flagged as a near tie.  Voxels touched by a near
tie in any frame are excluded from exact comparisons, since binary32 and
binary64 may legitimately decide them differently.
"""
from __future__ import annotations

import numpy as np

EPS_PX = 2e-3      # pixel-rounding margin (pixels)
EPS_M = 1e-5       # distance margin (metres)
EPS_F = 2e-5       # normalised TSDF margin
EPS_G = 1e-4       # grid-coordinate margin (voxels)


def _grid(dims, s, origin):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (origin[0] + (x + 0.5) * s, origin[1] + (y + 0.5) * s, origin[2] + (z + 0.5) * s)


def _to_camera(Twd, X, Y, Z):
    T = np.asarray(Twd, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    d = (X - t[0], Y - t[1], Z - t[2])
    # R^T (p - t)
    return tuple(R[0, r] * d[0] + R[1, r] * d[1] + R[2, r] * d[2] for r in range(3))


def _project(K, X, Y, Z):
    K = np.asarray(K, np.float64)
    xh = K[0, 0] * X + K[0, 1] * Y + K[0, 2] * Z
    yh = K[1, 0] * X + K[1, 1] * Y + K[1, 2] * Z
    zh = K[2, 0] * X + K[2, 1] * Y + K[2, 2] * Z
    ok = zh > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(ok, xh / np.where(ok, zh, 1.0), np.nan)
        v = np.where(ok, yh / np.where(ok, zh, 1.0), np.nan)
    tie = np.abs(zh) < 1e-6
    return u, v, ok, tie


def _round_tie(x):
    """True where x + 0.5 lies within EPS_PX of an integer (rounding ambiguity)."""
    f = np.mod(x + 0.5, 1.0)
    return (f < EPS_PX) | (f > 1 - EPS_PX)


def _nearest(u, v, ok, W, H):
    fu = np.floor(u + 0.5)
    fv = np.floor(v + 0.5)
    inside = ok & (fu >= 0) & (fu <= W - 1) & (fv >= 0) & (fv <= H - 1)
    tie = ok & (_round_tie(u) | _round_tie(v))
    iu = np.where(inside, fu, 0).astype(np.int64)
    iv = np.where(inside, fv, 0).astype(np.int64)
    return iu, iv, inside, tie


class Model:
    """Binary64 state of both volumes plus near-tie flags."""

    def __init__(self, dims_geo, dims_col, s_g, s_c, origin, mu, max_weight, sigma, band,
                 sample_mode=0, update_free_space=1):
        self.dg, self.dc = tuple(dims_geo), tuple(dims_col)
        self.s_g, self.s_c = float(s_g), float(s_c)
        self.o = tuple(float(v) for v in origin)
        self.mu, self.maxw = float(mu), int(max_weight)
        self.sigma, self.band = float(sigma), float(band)
        self.sample_mode, self.free = int(sample_mode), int(update_free_space)
        gshape = dims_geo[::-1]
        cshape = dims_col[::-1]
        self.F = np.zeros(gshape)
        self.W = np.zeros(gshape, np.int64)
        self.tie_g = np.zeros(gshape, bool)
        self.C = np.zeros(cshape + (3,), np.int64)
        self.CW = np.zeros(cshape, np.int64)
        self.tie_c = np.zeros(cshape, bool)

    # ---------------------------------------------------------------- TSDF
    def geometry(self, depth, Kd, Twd):
        H, W = depth.shape
        X, Y, Z = _to_camera(Twd, *_grid(self.dg, self.s_g, self.o))
        u, v, ok, tie0 = _project(Kd, X, Y, Z)
        iu, iv, inside, tie1 = _nearest(u, v, ok, W, H)
        D = np.where(inside, depth[iv, iu], 0).astype(np.float64)
        valid = inside & (D > 0)
        sdf = D * 1e-3 - Z
        upd = valid & (sdf >= -self.mu)
        tie = tie0 | tie1 | (valid & (np.abs(sdf + self.mu) < EPS_M))
        if not self.free:
            upd &= sdf <= self.mu
            tie |= valid & (np.abs(sdf - self.mu) < EPS_M)
        t = np.minimum(1.0, sdf / self.mu)
        Wf = self.W.astype(np.float64)
        self.F = np.where(upd, (self.F * Wf + t) / (Wf + 1.0), self.F)
        self.W = np.where(upd, np.minimum(self.W + 1, self.maxw), self.W)
        self.tie_g |= tie
        return upd

    # --------------------------------------------------------------- colour
    def _trilinear(self, gx, gy, gz):
        nx, ny, nz = self.dg
        g = (gx, gy, gz)
        i0 = [np.floor(a) for a in g]
        fr = [a - b for a, b in zip(g, i0)]
        tie = np.zeros(gx.shape, bool)
        inb = np.ones(gx.shape, bool)
        for a, n in zip(range(3), (nx, ny, nz)):
            inb &= (i0[a] >= 0) & (i0[a] + 1 <= n - 1)
            f = np.mod(g[a], 1.0)
            tie |= (f < EPS_G) | (f > 1 - EPS_G)
        ix = [np.clip(a, 0, n - 2).astype(np.int64) for a, n in zip(i0, (nx, ny, nz))]
        allw = inb.copy()
        anytie = np.zeros(gx.shape, bool)
        vals = {}
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    zz, yy, xx = ix[2] + dz, ix[1] + dy, ix[0] + dx
                    allw &= self.W[zz, yy, xx] > 0
                    anytie |= self.tie_g[zz, yy, xx]
                    vals[(dx, dy, dz)] = self.F[zz, yy, xx]
        fx, fy, fz = fr
        c00 = vals[0, 0, 0] + fx * (vals[1, 0, 0] - vals[0, 0, 0])
        c10 = vals[0, 1, 0] + fx * (vals[1, 1, 0] - vals[0, 1, 0])
        c01 = vals[0, 0, 1] + fx * (vals[1, 0, 1] - vals[0, 0, 1])
        c11 = vals[0, 1, 1] + fx * (vals[1, 1, 1] - vals[0, 1, 1])
        c0 = c00 + fy * (c10 - c00)
        c1 = c01 + fy * (c11 - c01)
        Ft = c0 + fz * (c1 - c0)
        return Ft, allw, tie | anytie

    def colour(self, depth, rgb, Kd, Kr, Twd, Tdr):
        H, W = depth.shape
        cH, cW, _ = rgb.shape
        Pw = _grid(self.dc, self.s_c, self.o)
        X, Y, Z = _to_camera(Twd, *Pw)
        u, v, ok, tie0 = _project(Kd, X, Y, Z)
        iu, iv, inside, tie1 = _nearest(u, v, ok, W, H)
        D = np.where(inside, depth[iv, iu], 0).astype(np.float64)
        valid = inside & (D > 0)
        d = D * 1e-3
        Kdi = np.linalg.inv(np.asarray(Kd, np.float64))
        q = [Kdi[r, 0] * iu + Kdi[r, 1] * iv + Kdi[r, 2] for r in range(3)]
        dist = np.sqrt((X - d * q[0]) ** 2 + (Y - d * q[1]) ** 2 + (Z - d * q[2]) ** 2)
        g_sigma = valid & (dist <= self.sigma)
        tie = tie0 | tie1 | (valid & (np.abs(dist - self.sigma) < EPS_M))
        g = [(Pw[a] - self.o[a]) / self.s_g - 0.5 for a in range(3)]
        Ft, allw, tie_t = self._trilinear(*g)
        g_band = allw & (np.abs(Ft) <= self.band)
        tie |= g_sigma & (tie_t | (allw & (np.abs(np.abs(Ft) - self.band) < EPS_F)))
        T = np.asarray(Tdr, np.float64)
        Xh = T[0, 0] * X + T[0, 1] * Y + T[0, 2] * Z + T[0, 3]
        Yh = T[1, 0] * X + T[1, 1] * Y + T[1, 2] * Z + T[1, 3]
        Zh = T[2, 0] * X + T[2, 1] * Y + T[2, 2] * Z + T[2, 3]
        uh, vh, okh, tie2 = _project(Kr, Xh, Yh, Zh)
        if self.sample_mode == 0:
            ju, jv, inh, tie3 = _nearest(uh, vh, okh, cW, cH)
            s = rgb[jv, ju].astype(np.int64)
        else:
            x0, y0 = np.floor(uh), np.floor(vh)
            inh = okh & (x0 >= 0) & (x0 + 1 <= cW - 1) & (y0 >= 0) & (y0 + 1 <= cH - 1)
            tie3 = okh & ((np.abs(uh - np.round(uh)) < EPS_PX) | (np.abs(vh - np.round(vh)) < EPS_PX))
            ax, ay = (uh - x0)[..., None], (vh - y0)[..., None]
            xi = np.where(inh, x0, 0).astype(np.int64)
            yi = np.where(inh, y0, 0).astype(np.int64)
            p00 = rgb[yi, xi].astype(np.float64)
            p10 = rgb[yi, np.minimum(xi + 1, cW - 1)].astype(np.float64)
            p01 = rgb[np.minimum(yi + 1, cH - 1), xi].astype(np.float64)
            p11 = rgb[np.minimum(yi + 1, cH - 1), np.minimum(xi + 1, cW - 1)].astype(np.float64)
            top = p00 + ax * (p10 - p00)
            bot = p01 + ax * (p11 - p01)
            val = top + ay * (bot - top)
            s = np.floor(val + 0.5).astype(np.int64)
            fr = np.mod(val + 0.5, 1.0)
            tie3 = tie3 | (inh & np.any((fr < 1e-3) | (fr > 1 - 1e-3), axis=-1))
        upd = g_sigma & g_band & inh
        tie |= g_sigma & g_band & (tie2 | tie3)
        w = self.CW[..., None]
        newc = (self.C * w + s + (w + 1) // 2) // (w + 1)
        self.C = np.where(upd[..., None], newc, self.C)
        self.CW = np.where(upd, np.minimum(self.CW + 1, self.maxw), self.CW)
        self.tie_c |= tie
        return upd

    def integrate(self, depth, rgb, Kd, Kr, Twd, Tdr):
        g = self.geometry(depth, Kd, Twd)
        c = self.colour(depth, rgb, Kd, Kr, Twd, Tdr)
        return g, c
