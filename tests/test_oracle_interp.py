"""Pins of the interpolated-heightmap oracle (Alg. 1, Sec. 3.3) against what geometry
and independent libraries fix: the triangulation equals Qhull's Delaunay triangulation
(scipy) for points in general position and has empty circumcircles; a linear height
field is reproduced exactly inside the convex hull; the nearest neighbour agrees with a
KD-tree (scipy) and breaks ties to the lowest index; texels outside the hull take the
nearest neighbour."""
import types

import numpy as np
import pytest
import scipy.spatial

from oracle import interp as I


def region(tiles=1):
    return types.SimpleNamespace(x0_cm=5_000_000, y0_cm=7_000_000, tile_cm=64000, tiles_x=tiles, tiles_y=tiles,
                                 z_scale=0.01, z_offset=0.0)


def samples_at(reg, lx, ly, z, rgb=None):
    n = len(lx)
    rgb = np.zeros((n, 3), np.int64) if rgb is None else rgb
    return {"x": np.asarray(lx, np.int64) + reg.x0_cm, "y": np.asarray(ly, np.int64) + reg.y0_cm,
            "z": np.asarray(z, np.int32), "r": rgb[:, 0].astype(np.uint16), "g": rgb[:, 1].astype(np.uint16),
            "b": rgb[:, 2].astype(np.uint16)}


def test_triangulation_equals_qhull_and_is_empty_circle():
    rng = np.random.default_rng(1)
    W = 96000
    pts = rng.integers(1, W, size=(80, 2))
    tris, V, ins = I.delaunay(pts, W)
    # Qhull on the same vertices (corners + points)
    allv = np.array(V, dtype=np.float64)
    q = scipy.spatial.Delaunay(allv)
    mine = {tuple(sorted(t)) for t in tris}
    theirs = {tuple(sorted(int(v) for v in s)) for s in q.simplices}
    assert mine == theirs
    # every triangle counter-clockwise and no vertex strictly inside a circumcircle
    for t in tris:
        a, b, c = (V[v] for v in t)
        assert I.orient(a, b, c) > 0
        for v in range(len(V)):
            if v not in t:
                assert I.incircle(a, b, c, V[v]) <= 0
    # Euler: 2 * n_vertices - 2 - hull vertices (the 4 corners) triangles
    assert len(tris) == 2 * len(V) - 2 - 4


def test_linear_field_is_reproduced_exactly_inside_the_hull():
    reg = region()
    rng = np.random.default_rng(2)
    lx = rng.integers(-10000, 74000, 60)
    ly = rng.integers(-10000, 74000, 60)
    z = 2 * (lx + 16000) + 3 * (ly + 16000) + 100  # linear in window coordinates, integer
    out = I.interp_tile(samples_at(reg, lx, ly, z), reg, 0)
    g = 1000 * np.arange(96) + 500
    GX, GY = np.meshgrid(g, g)
    plane = (2 * GX + 3 * GY + 100) * 0.01
    m = out["inside"] == 1
    assert m.sum() > 5000
    assert np.array_equal(out["lin_height"][m], plane[m])


def test_inside_is_covered_by_real_triangles_within_the_hull():
    """The linear map covers exactly the texels of the triangles of three real points
    (triangles with a corner padding point are the face map's -1, Alg. 1): checked on
    Qhull's triangulation of corners + points, and always inside the convex hull of
    the real points (padding triangles may reach into that hull near its boundary)."""
    reg = region()
    rng = np.random.default_rng(3)
    lx = rng.integers(0, 64000, 40)
    ly = rng.integers(0, 64000, 40)
    out = I.interp_tile(samples_at(reg, lx, ly, rng.integers(-500, 500, 40)), reg, 0)
    P = np.stack([lx + 16000, ly + 16000], -1)
    g = 1000 * np.arange(96) + 500
    GX, GY = np.meshgrid(g, g)
    corners = np.array([[0, 0], [96000, 0], [96000, 96000], [0, 96000]])
    allv = np.concatenate([corners, P]).astype(np.int64)
    q = scipy.spatial.Delaunay(allv.astype(np.float64))
    cover = np.zeros((96, 96), bool)
    for sx in q.simplices:
        if min(sx) < 4:
            continue
        a, b, c = (allv[v] for v in sx)
        if I.orient(a, b, c) < 0:
            b, c = c, b
        wa = (b[0] - GX) * (c[1] - GY) - (b[1] - GY) * (c[0] - GX)
        wb = (c[0] - GX) * (a[1] - GY) - (c[1] - GY) * (a[0] - GX)
        wc = (a[0] - GX) * (b[1] - GY) - (a[1] - GY) * (b[0] - GX)
        cover |= (wa >= 0) & (wb >= 0) & (wc >= 0)
    assert np.array_equal(out["inside"].astype(bool), cover)
    hull = scipy.spatial.Delaunay(P.astype(np.float64))
    inhull = (hull.find_simplex(np.stack([GX.ravel(), GY.ravel()], -1).astype(np.float64)) >= 0).reshape(96, 96)
    assert not (cover & ~inhull).any()
    assert cover.sum() > 0.95 * inhull.sum()
    # outside the real triangles the linear map is the nearest-neighbour map
    o = out["inside"] == 0
    assert np.array_equal(out["lin_height"][o], out["nn_height"][o])


def test_nearest_neighbour_matches_kdtree_and_ties_go_to_lowest_index():
    reg = region()
    rng = np.random.default_rng(4)
    lx = rng.integers(-16000, 80000, 200)
    ly = rng.integers(-16000, 80000, 200)
    z = rng.integers(-9000, 9000, 200)
    out = I.interp_tile(samples_at(reg, lx, ly, z), reg, 0)
    P = np.stack([lx + 16000, ly + 16000], -1)
    g = 1000 * np.arange(96) + 500
    GX, GY = np.meshgrid(g, g)
    tree = scipy.spatial.cKDTree(P.astype(np.float64))
    dist, idx = tree.query(np.stack([GX.ravel(), GY.ravel()], -1).astype(np.float64))
    kd_h = (z[idx] * 0.01).reshape(96, 96)
    # where the KD-tree's choice is the unique nearest point, heights agree exactly
    d2 = (GX[..., None] - P[:, 0]) ** 2 + (GY[..., None] - P[:, 1]) ** 2
    unique = (d2 == d2.min(-1, keepdims=True)).sum(-1) == 1
    assert unique.mean() > 0.99
    assert np.array_equal(out["nn_height"][unique], kd_h[unique])
    # hand-made tie: two points at the same distance from texel (0, 0) -> lower index
    s = samples_at(reg, [-16000 + 500 - 300, -16000 + 500 + 300], [-16000 + 500, -16000 + 500], [111, 222])
    o2 = I.interp_tile(s, reg, 0)
    assert o2["nn_height"][0, 0] == pytest.approx(1.11)


def test_duplicates_skipped_and_empty_window():
    reg = region()
    lx = np.array([1000, 1000, 30000, 50000, 5000])
    ly = np.array([1000, 1000, 40000, 2000, 60000])
    tris, V, ins = I.delaunay(np.stack([lx, ly], -1), 96000)
    assert len(ins) == 4  # the duplicate is not a vertex
    out = I.interp_tile(samples_at(reg, [200000], [200000], [5]), reg, 0)  # outside the window
    assert np.isnan(out["nn_height"]).all() and np.isnan(out["lin_height"]).all()
    assert (out["inside"] == 0).all()


def test_constant_heights_fill_exactly():
    reg = region()
    rng = np.random.default_rng(6)
    lx = rng.integers(-16000, 80000, 50)
    ly = rng.integers(-16000, 80000, 50)
    out = I.interp_tile(samples_at(reg, lx, ly, np.full(50, 4321)), reg, 0)
    assert np.all(out["lin_height"] == 43.21) and np.all(out["nn_height"] == 43.21)
