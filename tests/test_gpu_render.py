"""GPU parity of the software rasterizers against the oracle: framebuffers bit-exact
(every 64-bit word), resolve bit-exact, for points and heightmap meshes under oblique
perspective and close-up cameras (large triangles through the CTA queue), with holes."""
import numpy as np
import pytest

import oracle.render as R
import synth
from tests.helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


def look_at(eye, target, up=(0.0, 0.0, 1.0), fovy_deg=60.0, aspect=1.0, near=100.0, far=1e7):
    """OpenGL-style view-projection (row-major, float32) for a camera at `eye` (cm, in
    the camera frame whose origin is the camera's integer origin)."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = s, u, -f
    V[:3, 3] = -V[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    P = np.zeros((4, 4))
    P[0, 0], P[1, 1] = t / aspect, t
    P[2, 2], P[2, 3] = (far + near) / (near - far), 2 * far * near / (near - far)
    P[3, 2] = -1.0
    return (P @ V).astype(np.float32).ravel().tolist()


def camera(region, eye_m, target_m, width, height, fovy=60.0, near=100.0):
    """Camera with its integer origin at the region's south-west corner."""
    o = (region.x0_cm, region.y0_cm, 0)
    return {"origin_cm": o, "width": width, "height": height,
            "view_proj": look_at(np.asarray(eye_m) * 100, np.asarray(target_m) * 100, fovy_deg=fovy,
                                 aspect=width / height, near=near)}


def gpu_fb(lsb, cam):
    return lsb.render_framebuffer(cam)


def as_u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_points_oblique_perspective(lsb):
    import torch
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = np.full(9, 40_000, np.int64)
    pts = synth.region_points(4, region, counts)
    del pts["tile_offsets"]
    cam = camera(region, (-300, -500, 900), (960, 960, 400), 320, 240)
    fb = gpu_fb(lsb, cam)
    lsb.render_points(to_device(pts), cam, fb)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    ref = R.render_points(R.clear(320, 240), pts, cam)
    np.testing.assert_array_equal(as_u64(fb), ref)
    assert (ref != R.EMPTY).sum() > 5000
    img = lsb.render_resolve(fb, background=0xFF332211)
    np.testing.assert_array_equal(img.cpu().numpy(), R.resolve(ref, 0xFF332211))


def test_points_top_down_dense_ties(lsb):
    """Many points per pixel (depth ties decided by the colour word)."""
    import torch
    region = synth.Region(tiles_x=1, tiles_y=1)
    rng = np.random.default_rng(3)
    n = 300_000
    p = {"x": region.x0_cm + rng.integers(0, 64000, n), "y": region.y0_cm + rng.integers(0, 64000, n),
         "z": rng.integers(0, 4, n), "r": rng.integers(0, 65536, n), "g": rng.integers(0, 65536, n),
         "b": rng.integers(0, 65536, n)}
    p = {k: v.astype(np.int32 if k in "xyz" else np.uint16) for k, v in p.items()}
    M = [2.0 ** -15, 0, 0, -1, 0, 2.0 ** -15, 0, -1, 0, 0, 2.0 ** -13, -1, 0, 0, 0, 1]
    cam = {"origin_cm": (region.x0_cm, region.y0_cm, 0), "view_proj": M, "width": 64, "height": 64}
    fb = gpu_fb(lsb, cam)
    lsb.render_points(to_device(p), cam, fb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(as_u64(fb), R.render_points(R.clear(64, 64), p, cam))


def _heightmaps(lsb, region, res, seed=6):
    counts = synth.lognormal_counts(seed, region.n_tiles)
    s = synth.region_samples(seed, region, counts)
    h, c = lsb.fill_sparse(to_device(s), region, res=res)
    return h, c


@pytest.mark.parametrize("view", ["oblique", "close"])
def test_heightmap_meshes(lsb, view):
    import torch
    region = synth.Region(tiles_x=3, tiles_y=2, z_offset=12.5)
    res = 32
    h, c = _heightmaps(lsb, region, res)
    h[1, 10:14, 5:9] = float("nan")  # a hole
    if view == "oblique":
        cam = camera(region, (-400, -600, 1500), (960, 640, 350), 400, 300)
    else:  # 30 m over the terrain: near triangles cover thousands of pixels
        z = float(h[1, 15, 3]) - region.z_offset
        cam = camera(region, (700, 300, z + 30), (760, 340, z - 10), 256, 256, fovy=90.0)
    tiles = torch.tensor([0, 1, 2, 3, 4, 5], dtype=torch.int32)
    fb = gpu_fb(lsb, cam)
    lsb.render_heightmaps(h, c, region, cam, fb, tile_ids=tiles)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    ref = R.render_heightmaps(R.clear(cam["width"], cam["height"]), h.cpu().numpy(), c.cpu().numpy(),
                              range(6), region, cam)
    np.testing.assert_array_equal(as_u64(fb), ref)
    assert (ref != R.EMPTY).sum() > 1000
    if view == "close":
        # some triangle has more than 1024 candidate pixels (the CTA-queue path ran)
        assert _largest_candidate_box(h.cpu().numpy(), region, cam) > 1024


def _largest_candidate_box(h, region, cam):
    best = 0
    for o in range(h.shape[0]):
        q, has = R.heightmap_vertices(h[o], region, o, cam)
        sx, sy, d, kept = R._project(q.reshape(-1, 3), cam["view_proj"], cam["width"], cam["height"])
        ok = kept & has.reshape(-1)
        res = h.shape[1]
        sx, sy, ok = sx.reshape(res, res), sy.reshape(res, res), ok.reshape(res, res)
        for i in range(res - 1):
            for j in range(res - 1):
                if ok[i, j] and ok[i + 1, j + 1] and ok[i, j + 1]:
                    xs = [sx[i, j], sx[i, j + 1], sx[i + 1, j + 1]]
                    ys = [sy[i, j], sy[i, j + 1], sy[i + 1, j + 1]]
                    xa, xb = max(0, int(np.floor(min(xs)))), min(cam["width"] - 1, int(np.floor(max(xs))))
                    ya, yb = max(0, int(np.floor(min(ys)))), min(cam["height"] - 1, int(np.floor(max(ys))))
                    if xb >= xa and yb >= ya:
                        best = max(best, (xb - xa + 1) * (yb - ya + 1))
    return best


def test_points_over_heightmaps_and_order_independence(lsb):
    """Points and meshes into one framebuffer, in both orders: the same words."""
    import torch
    region = synth.Region(tiles_x=2, tiles_y=2)
    res = 16
    h, c = _heightmaps(lsb, region, res, seed=7)
    counts = synth.lognormal_counts(7, 4)
    s = synth.region_samples(7, region, counts)
    cam = camera(region, (-200, -200, 800), (640, 640, 350), 200, 160)
    a = gpu_fb(lsb, cam)
    lsb.render_heightmaps(h, c, region, cam, a)
    lsb.render_points(to_device(s), cam, a)
    b = gpu_fb(lsb, cam)
    lsb.render_points(to_device(s), cam, b)
    lsb.render_heightmaps(h, c, region, cam, b)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(as_u64(a), as_u64(b))
    ref = R.render_heightmaps(R.clear(200, 160), h.cpu().numpy(), c.cpu().numpy(), range(4), region, cam)
    ref = R.render_points(ref, s, cam)
    np.testing.assert_array_equal(as_u64(a), ref)


def test_points_unaligned_arrays_and_tail(lsb):
    """Arrays that are not 16-byte aligned (the point-by-point path) and a count that is
    not a multiple of 4 (the tail of the vector path)."""
    import torch
    region = synth.Region(tiles_x=2, tiles_y=1)
    pts = synth.region_points(5, region, np.array([30_001, 20_002], np.int64))
    del pts["tile_offsets"]
    cam = camera(region, (-100, -300, 700), (640, 320, 400), 160, 120)
    d = to_device(pts)
    ref = R.render_points(R.clear(160, 120), {k: v[1:] for k, v in pts.items()}, cam)
    for sub in ({k: v[1:] for k, v in d.items()},                      # 4-byte aligned only
                {k: v[1:].clone() for k, v in d.items()}):             # aligned, n % 4 == 2
        fb = gpu_fb(lsb, cam)
        lsb.render_points(sub, cam, fb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(as_u64(fb), ref)
