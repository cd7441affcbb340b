"""Oracle of the interpolated heightmaps of Alg. 1 (Sec. 3.3): nearest-neighbour and
Delaunay-linear heightmaps of a padded patch (TEST INFRASTRUCTURE ONLY: imported by
tests/ and nothing in the product path).

The patch of tile t is the window of side W = tile + 2 * pad around the tile (the
paper's 96 x 96 texels of 10 m for a 64 x 64 tile, the padding avoiding seams between
neighbouring patches, Sec. 3.3).  Window-local integer centimetres replace the paper's
[-1, 1]^2 patch space (an affine map, which changes neither the triangulation nor the
interpolated values).  Steps, in the order of Alg. 1:

1. points: the chunk samples inside the closed window, in global sample order;
2. four corner padding points (no data) at the window corners, then the Delaunay
   triangulation of corners and points (Bowyer-Watson, exact integer predicates);
3. every grid point (texel centre) inside a triangle whose three vertices are real
   points gets the linear (barycentric) interpolation of that triangle; the others,
   and all texels of the NN map, get the nearest point's values.

The face map of Alg. 1 (a flood fill from triangle centroids, then from the pixels of
each triangle's bounding box) is the way the paper finds, for every texel, the
triangle that contains it; here every texel is tested against every triangle, which
reaches the same containing triangle.  Exact integer arithmetic makes the result
independent of the order of those tests: on an edge shared by two real triangles both
give the same rational value, and the division is the only rounding.
"""
from __future__ import annotations

import numpy as np


def orient(a, b, c):
    """Twice the signed area of (a, b, c); > 0 for counter-clockwise."""
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def incircle(a, b, c, d):
    """> 0 iff d lies strictly inside the circumcircle of the counter-clockwise
    triangle (a, b, c) (the standard lifted 3x3 determinant, exact integers)."""
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    ad = adx * adx + ady * ady
    bd = bdx * bdx + bdy * bdy
    cd = cdx * cdx + cdy * cdy
    return (adx * (bdy * cd - bd * cdy) - ady * (bdx * cd - bd * cdx) + ad * (bdx * cdy - bdy * cdx))


def delaunay(pts, W):
    """Bowyer-Watson triangulation of the square [0, W]^2's corners (vertices 0..3)
    followed by pts (vertices 4.., inserted in order).  A point equal to an earlier
    vertex is skipped.  A triangle is "bad" for a new point when the point lies strictly
    inside its circumcircle; the cavity's boundary edges are joined to the point
    (degenerate, zero-area joins on the square's edges are dropped).  Returns the list
    of counter-clockwise vertex triples and the list of inserted vertex ids."""
    V = [(0, 0), (W, 0), (W, W), (0, W)] + [tuple(int(v) for v in p) for p in pts]
    tris = [(0, 1, 2), (0, 2, 3)]
    seen = {V[0]: 0, V[1]: 1, V[2]: 2, V[3]: 3}
    inserted = []
    for vi in range(4, len(V)):
        p = V[vi]
        if p in seen:
            continue
        seen[p] = vi
        bad = [t for t in tris if incircle(V[t[0]], V[t[1]], V[t[2]], p) > 0]
        count = {}
        for t in bad:
            for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
                key = (min(e), max(e))
                count[key] = count.get(key, 0) + 1
        badset = set(bad)
        tris = [t for t in tris if t not in badset]
        for t in bad:
            for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
                if count[(min(a, b), max(a, b))] == 1 and orient(V[a], V[b], p) > 0:
                    tris.append((a, b, vi))
        inserted.append(vi)
    return tris, V, inserted


def window_of(region, t, pad_cm):
    tx, ty = t % region.tiles_x, t // region.tiles_x
    return tx * region.tile_cm - pad_cm, ty * region.tile_cm - pad_cm, region.tile_cm + 2 * pad_cm


def interp_tile(samples, region, t, res=96, pad_cm=16000):
    """Alg. 1 for tile t.  Returns dict: nn_height, lin_height float64 [res, res] (m),
    nn_rgb8, lin_rgb8 float64 [res, res, 3] (8-bit scale, unrounded), inside uint8
    [res, res] (1 where the linear map interpolates), triangles (list of triples of
    global sample indices, -1 - c for corner c: 0 = (0, 0), 1 = (W, 0), 2 = (W, W),
    3 = (0, W) in window coordinates)."""
    X0, Y0, W = window_of(region, t, pad_cm)
    assert W % res == 0
    # the int64 numerators below (weights up to W^2 times heights) stay exact for
    # |z| < 2^28 cm (2,680 km)
    assert len(samples["z"]) == 0 or int(np.abs(samples["z"].astype(np.int64)).max()) < 2 ** 28
    cell = W // res
    lx = samples["x"].astype(np.int64) - region.x0_cm - X0
    ly = samples["y"].astype(np.int64) - region.y0_cm - Y0
    sel = np.nonzero((lx >= 0) & (lx <= W) & (ly >= 0) & (ly <= W))[0]
    pts = [(int(lx[i]), int(ly[i])) for i in sel]
    z = samples["z"].astype(np.int64)[sel]
    rgb = np.stack([samples[k].astype(np.int64)[sel] for k in "rgb"], -1) if len(sel) else np.zeros((0, 3), np.int64)
    tris, V, _ = delaunay(pts, W)
    out = {"nn_height": np.full((res, res), np.nan), "lin_height": np.full((res, res), np.nan),
           "nn_rgb8": np.zeros((res, res, 3)), "lin_rgb8": np.zeros((res, res, 3)),
           "inside": np.zeros((res, res), np.uint8),
           "triangles": [tuple(int(sel[v - 4]) if v >= 4 else -1 - v for v in tr) for tr in tris]}
    gx = cell * np.arange(res, dtype=np.int64) + cell // 2
    GX, GY = np.meshgrid(gx, gx)  # [i][j]: GX column j, GY row i
    # nearest point (exact int64 squared distance; ties to the lowest sample index)
    if len(sel):
        P = np.array(pts, dtype=np.int64)
        k = np.empty((res, res), dtype=np.int64)
        for i in range(res):  # one texel row at a time (memory res x n at any res)
            d2 = (gx[:, None] - P[:, 0]) ** 2 + (gx[i] - P[:, 1]) ** 2
            k[i] = np.argmin(d2, axis=-1)  # first minimum = lowest index (sel is increasing)
        out["nn_height"] = z[k] * region.z_scale + region.z_offset
        out["nn_rgb8"] = rgb[k] / 256.0
        out["lin_height"] = out["nn_height"].copy()
        out["lin_rgb8"] = out["nn_rgb8"].copy()
    # linear interpolation in triangles of three real points
    for tr in tris:
        if min(tr) < 4:
            continue
        a, b, c = (V[v] for v in tr)
        A = orient(a, b, c)
        wa = (b[0] - GX) * (c[1] - GY) - (b[1] - GY) * (c[0] - GX)
        wb = (c[0] - GX) * (a[1] - GY) - (c[1] - GY) * (a[0] - GX)
        wc = (a[0] - GX) * (b[1] - GY) - (a[1] - GY) * (b[0] - GX)
        m = (wa >= 0) & (wb >= 0) & (wc >= 0)
        if not m.any():
            continue
        ia, ib, ic = (v - 4 for v in tr)
        num = wa[m] * z[ia] + wb[m] * z[ib] + wc[m] * z[ic]
        out["lin_height"][m] = num / A * region.z_scale + region.z_offset
        for ch in range(3):
            numc = wa[m] * rgb[ia, ch] + wb[m] * rgb[ib, ch] + wc[m] * rgb[ic, ch]
            out["lin_rgb8"][..., ch][m] = numc / A / 256.0
        out["inside"][m] = 1
    return out
