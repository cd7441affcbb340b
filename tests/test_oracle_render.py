"""Pins of the rasterizer oracle (oracle/render.py) against hand-computed pixels and
closed-form coverage: an orthographic top-down camera whose scales are powers of two
makes every projected coordinate exact, so pixels, depths and covered pixel sets follow
from integer arithmetic."""
import numpy as np

import oracle.render as R
import synth

W = H = 64
# camera frame (cm) x, y in [0, 8192) -> ndc [-1, 1): 128 cm per pixel; depth d = z / 2^14
ORTHO = [2.0 ** -12, 0, 0, -1,
         0, 2.0 ** -12, 0, -1,
         0, 0, 2.0 ** -13, -1,
         0, 0, 0, 1]


def cam(origin=(0, 0, 0), M=ORTHO):
    return {"origin_cm": origin, "view_proj": M, "width": W, "height": H}


def word(d, r, g, b):
    bits = np.array([d], np.float32).view(np.uint32)[0]
    return (int(bits) << 32) | r | (g << 8) | (b << 16) | (255 << 24)


def pts(xyz, rgb16):
    xyz = np.asarray(xyz, np.int64)
    rgb16 = np.asarray(rgb16, np.int64)
    return {"x": xyz[:, 0], "y": xyz[:, 1], "z": xyz[:, 2], "r": rgb16[:, 0], "g": rgb16[:, 1], "b": rgb16[:, 2]}


def test_points_land_on_hand_computed_pixels_nearest_wins():
    p = pts([(300, 200, 1024),     # pixel (2, 1), d = 1024 / 16384
             (300 + 10, 250, 512),  # same pixel, nearer: wins
             (8191, 8191, 0),      # last pixel, d = 0
             (-1, 5, 10),          # left of the screen: dropped
             (5, 5, 16385),        # d > 1: dropped
             (1000, 1000, 2048),   # pixel (7, 7)
             (1001, 1001, 2048)],  # same pixel, same depth, smaller colour word wins
            [(65535, 0, 0), (0, 256, 0), (128, 127, 383), (1, 1, 1), (1, 1, 1), (512, 0, 0), (256, 0, 0)])
    fb = R.render_points(R.clear(W, H), p, cam())
    assert fb[1, 2] == word(512 / 16384, 0, 1, 0)
    assert fb[63, 63] == word(0.0, 1, 0, 1)  # (128 + 128) >> 8 = 1, 127 + 128 >> 8 = 0, (383+128)>>8 = 1
    assert fb[7, 7] == word(2048 / 16384, 1, 0, 0)
    covered = fb != R.EMPTY
    assert covered.sum() == 3


def test_camera_origin_and_behind_the_camera():
    o = (50_000_000, 400_000_000, 1000)
    p = pts([(o[0] + 300, o[1] + 200, o[2] + 1024)], [(0, 0, 0)])
    fb = R.render_points(R.clear(W, H), p, cam(origin=o))
    assert fb[1, 2] == word(1024 / 16384, 0, 0, 0)
    flip = list(ORTHO)
    flip[15] = -1.0  # c_w < 0: behind the camera
    assert (R.render_points(R.clear(W, H), p, cam(origin=o, M=flip)) == R.EMPTY).all()


def test_perspective_point_straight_ahead_hits_the_centre():
    # camera looking along +x from the origin: ndc_x = y / x, ndc_y = z / x, c_w = x
    f = 1.0
    M = [0, f, 0, 0,
         0, 0, f, 0,
         0.5, 0, 0, 0,   # c_z = x / 2: d = 0.75 for any x > 0
         1, 0, 0, 0]
    p = pts([(1000, 0, 0), (5000, 1, 1)], [(0, 0, 0), (256, 256, 256)])
    fb = R.render_points(R.clear(W, H), p, cam(M=M))
    assert fb[32, 32] == word(0.75, 0, 0, 0)  # equal depths: the smaller colour word


def _tri_fb(v, col):
    fb = R.clear(W, H)
    R.draw_triangle(fb, np.asarray(v, np.float32), np.asarray(col, np.float32))
    return fb


def test_right_triangle_covers_the_closed_form_pixel_set():
    # vertices at screen (0, 0), (64, 0), (0, 64): pixel centre (i + .5, j + .5) covered
    # iff i + j + 1 <= 64, i.e. i + j <= 63: 64 * 65 / 2 pixels
    for order in ((0, 1, 2), (0, 2, 1)):  # both orientations
        v = np.array([(0, 0, 0.25), (64, 0, 0.25), (0, 64, 0.25)], np.float32)[list(order)]
        fb = _tri_fb(v, [(10, 20, 30)] * 3)
        cov = fb != R.EMPTY
        i, j = np.meshgrid(np.arange(W), np.arange(H))
        np.testing.assert_array_equal(cov, (i + j) <= 63)
        assert (fb[cov] == word(0.25, 10, 20, 30)).all()


def test_colour_and_depth_interpolate_linearly():
    # screen triangle (0,0), (64,0), (0,64); depth d = 0.5 x / 64 and red = 4 * y at
    # pixel centres (dyadic weights: exact in float)
    v = [(0, 0, 0.0), (64, 0, 0.5), (0, 64, 0.0)]
    col = [(0, 0, 0), (0, 0, 0), (256, 0, 0)]
    fb = _tri_fb(v, col)
    for (x, y) in [(0, 0), (10, 5), (31, 31), (62, 1)]:
        d = 0.5 * (x + 0.5) / 64
        red = min(255, int(np.floor(256 * (y + 0.5) / 64 + 0.5)))
        assert fb[y, x] == word(d, red, 0, 0), (x, y)


def test_flat_heightmap_covers_its_texel_centre_square_and_holes():
    # one 640 m tile, res 8 (80 m texels): texel centres at 40 m + 80 m j, i.e. camera
    # x = 4000 + 8000 j cm; with 2^-15 in M (1024 cm per pixel at 64 pixels) the square between the
    # first and last centres spans x in [4000, 60000] cm = [3.906, 58.59] pixels
    region = synth.Region(x0_cm=0, y0_cm=0, tiles_x=1, tiles_y=1, z_offset=0.0)
    M = [2.0 ** -15, 0, 0, -1, 0, 2.0 ** -15, 0, -1, 0, 0, 2.0 ** -13, -1, 0, 0, 0, 1]
    res = 8
    h = np.full((1, res, res), 20.48, np.float32)  # 2048 cm: d = 0.125
    rgb = np.zeros((1, res, res, 3), np.uint8)
    rgb[..., 1] = 200
    fb = R.render_heightmaps(R.clear(W, H), h, rgb, [0], region, cam(M=M))
    cov = fb != R.EMPTY
    c = np.arange(W) + 0.5
    inside = (c >= 4000 / 1024) & (c <= 60000 / 1024)
    np.testing.assert_array_equal(cov, inside[:, None] & inside[None, :])
    zb = np.float32(np.float32(20.48) * np.float32(100.0))  # the height in cm, as computed
    d = np.float32(np.float32(zb * np.float32(2.0 ** -13) - 1) * np.float32(0.5) + np.float32(0.5))
    # colour exact; depth: the constant times the rounded sum of the three weights
    assert ((fb[cov] & np.uint64(0xFFFFFFFF)) == (200 << 8) | (255 << 24)).all()
    depth = (fb[cov] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.abs(depth - d).max() <= 4 * np.spacing(d)
    # a NaN texel removes the triangles of its quads
    h[0, 3, 3] = np.nan
    fb2 = R.render_heightmaps(R.clear(W, H), h, rgb, [0], region, cam(M=M))
    hole = cov & (fb2 == R.EMPTY)
    cx = (4000 + 8000 * np.arange(res)) / 1024
    ys, xs = np.nonzero(hole)
    assert hole.sum() > 0
    assert (c[xs] > cx[2]).all() and (c[xs] < cx[4]).all() and (c[ys] > cx[2]).all() and (c[ys] < cx[4]).all()


def test_resolve():
    fb = R.clear(4, 2)
    fb[0, 1] = word(0.5, 1, 2, 3)
    img = R.resolve(fb, 0x80402010)
    assert tuple(img[0, 1]) == (1, 2, 3, 255)
    assert tuple(img[1, 3]) == (0x10, 0x20, 0x40, 0x80)
