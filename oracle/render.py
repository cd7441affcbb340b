"""Oracle of the software rasterizers (Sec. 3.5, rendering): points and heightmap
triangles into a 64-bit depth|colour framebuffer, smallest word per pixel, and the
resolve into RGBA8 (TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing in the
product path).

Every float operation is a numpy float32 operation (one IEEE rounding each, no fused
multiply-add), in the order the rasterizer's definition fixes:

  camera frame  q = ((f32)(x - ox), (f32)(y - oy), (f32)(z - oz)) in cm
  clip          c_r = ((M[r,0] q.x + M[r,1] q.y) + M[r,2] q.z) + M[r,3]
  kept          c_w > 0, ndc = c / c_w, d = ndc_z * 0.5 + 0.5 in [0, 1]
  screen        sx = (ndc_x * 0.5 + 0.5) * width, sy = (ndc_y * 0.5 + 0.5) * height
  word          bits(d) << 32 | R | G << 8 | B << 16 | 255 << 24

Points land on pixel (floor(sx), floor(sy)).  A triangle covers the pixel centres where
its three edge functions (signs normalised by the signed area) are >= 0, with depth and
colour interpolated by the barycentric weights e_k / A.  The framebuffer keeps the
minimum word of each pixel (np.minimum.at), which makes it independent of the order in
which fragments arrive.
"""
from __future__ import annotations

import numpy as np

F = np.float32
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def clear(width, height):
    return np.full((height, width), EMPTY, dtype=np.uint64)


def _project(q, M, width, height):
    """q: float32 [n, 3].  Returns sx, sy, d (float32) and the kept mask."""
    M = np.asarray(M, dtype=F).reshape(4, 4)
    c = [((M[r, 0] * q[:, 0] + M[r, 1] * q[:, 1]) + M[r, 2] * q[:, 2]) + M[r, 3] for r in range(4)]
    cw = c[3]
    with np.errstate(divide="ignore", invalid="ignore"):
        ndc = [c[k] / cw for k in range(3)]  # the perspective division, one IEEE quotient each
    half = F(0.5)
    sx = (ndc[0] * half + half) * F(width)
    sy = (ndc[1] * half + half) * F(height)
    d = ndc[2] * half + half
    kept = (cw > 0) & (d >= 0) & (d <= 1) & np.isfinite(sx) & np.isfinite(sy)
    return sx, sy, d, kept


def _word(d, r8, g8, b8):
    bits = d.astype(F).view(np.uint32).astype(np.uint64)
    col = (r8.astype(np.uint64) | (g8.astype(np.uint64) << np.uint64(8)) | (b8.astype(np.uint64) << np.uint64(16))
           | np.uint64(255 << 24))
    return (bits << np.uint64(32)) | col


def to8(c16):
    """16-bit colour to 8 bits, round half up, clamped."""
    return np.minimum((np.asarray(c16, np.int64) + 128) >> 8, 255)


def render_points(fb, pts, camera):
    """pts: dict of x, y, z (LAS integers) and r, g, b (16-bit); camera: dict with
    origin_cm (3 ints), view_proj (16 floats, row-major), width, height."""
    W, H = camera["width"], camera["height"]
    o = camera["origin_cm"]
    q = np.stack([(np.asarray(pts[k], np.int64) - int(o[i])).astype(F) for i, k in enumerate("xyz")], -1)
    sx, sy, d, kept = _project(q, camera["view_proj"], W, H)
    with np.errstate(invalid="ignore"):
        ix = np.floor(sx)
        iy = np.floor(sy)
    on = kept & (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
    w = _word(d[on], to8(pts["r"])[on], to8(pts["g"])[on], to8(pts["b"])[on])
    np.minimum.at(fb, (iy[on].astype(np.int64), ix[on].astype(np.int64)), w)
    return fb


def heightmap_vertices(height, region, t, camera):
    """Camera-frame vertices (float32 [res, res, 3]) of the texel centres of tile t and
    the mask of texels with a height."""
    res = height.shape[0]
    cell = region.tile_cm // res
    tx, ty = t % region.tiles_x, t // region.tiles_x
    o = camera["origin_cm"]
    j = np.arange(res, dtype=np.int64)
    xs = region.x0_cm + tx * region.tile_cm + cell * j + cell // 2
    ys = region.y0_cm + ty * region.tile_cm + cell * j + cell // 2
    qx = (xs - int(o[0])).astype(F)
    qy = (ys - int(o[1])).astype(F)
    izs = F(1.0 / region.z_scale)
    qz = ((height.astype(F) - F(region.z_offset)) * izs) - F(int(o[2]))
    q = np.empty((res, res, 3), F)
    q[..., 0] = qx[None, :]
    q[..., 1] = qy[:, None]
    q[..., 2] = qz
    return q, ~np.isnan(height)


def draw_triangle(fb, v, col):
    """v: float32 [3, 3] screen (sx, sy, d) of the three vertices; col: float32 [3, 3]
    8-bit vertex colours.  Draws the covered pixels."""
    H, W = fb.shape
    x0, y0 = v[0, 0], v[0, 1]
    x1, y1 = v[1, 0], v[1, 1]
    x2, y2 = v[2, 0], v[2, 1]
    A = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0)
    if not np.isfinite(A) or A == 0:
        return
    ixa = max(0, int(np.floor(min(x0, x1, x2))))
    ixb = min(W - 1, int(np.floor(max(x0, x1, x2))))
    iya = max(0, int(np.floor(min(y0, y1, y2))))
    iyb = min(H - 1, int(np.floor(max(y0, y1, y2))))
    if ixa > ixb or iya > iyb:
        return
    px = np.arange(ixa, ixb + 1).astype(F) + F(0.5)
    py = np.arange(iya, iyb + 1).astype(F) + F(0.5)
    PX, PY = np.meshgrid(px, py)
    e0 = (x2 - x1) * (PY - y1) - (y2 - y1) * (PX - x1)
    e1 = (x0 - x2) * (PY - y2) - (y0 - y2) * (PX - x2)
    e2 = (x1 - x0) * (PY - y0) - (y1 - y0) * (PX - x0)
    if A < 0:
        e0, e1, e2, A = -e0, -e1, -e2, -A
    m = (e0 >= 0) & (e1 >= 0) & (e2 >= 0)
    if not m.any():
        return
    l0, l1, l2 = e0[m] / A, e1[m] / A, e2[m] / A
    d = (l0 * v[0, 2] + l1 * v[1, 2]) + l2 * v[2, 2]
    ch = []
    for k in range(3):
        c = ((l0 * col[0, k] + l1 * col[1, k]) + l2 * col[2, k]) + F(0.5)
        ch.append(np.clip(np.floor(c), 0, 255).astype(np.int64))
    w = _word(d, ch[0], ch[1], ch[2])
    iy, ix = np.nonzero(m)
    np.minimum.at(fb, (iy + iya, ix + ixa), w)


def render_heightmaps(fb, height, rgb, tile_ids, region, camera):
    """height float32 [n, res, res] (metres, NaN = no data), rgb uint8 [n, res, res, 3];
    two triangles per quad of adjacent texel centres: (v00, v01, v11), (v00, v11, v10)."""
    W, H = camera["width"], camera["height"]
    for o, t in enumerate(tile_ids):
        q, has = heightmap_vertices(np.asarray(height[o], F), region, int(t), camera)
        res = q.shape[0]
        sx, sy, d, kept = _project(q.reshape(-1, 3), camera["view_proj"], W, H)
        ok = (kept & has.reshape(-1)).reshape(res, res)
        S = np.stack([sx, sy, d], -1).reshape(res, res, 3)
        C = np.asarray(rgb[o]).astype(F)
        for i in range(res - 1):
            for j in range(res - 1):
                quad = [(i, j), (i, j + 1), (i + 1, j + 1), (i + 1, j)]
                for tri in ((0, 1, 2), (0, 2, 3)):
                    vs = [quad[k] for k in tri]
                    if all(ok[a, b] for a, b in vs):
                        draw_triangle(fb, np.stack([S[a, b] for a, b in vs]), np.stack([C[a, b] for a, b in vs]))
    return fb


def resolve(fb, background):
    """RGBA8 [H, W, 4]: the colour word of covered pixels, background elsewhere."""
    low = (fb & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out = np.where(fb == EMPTY, np.uint32(background), low)
    return out.view(np.uint8).reshape(fb.shape + (4,))
