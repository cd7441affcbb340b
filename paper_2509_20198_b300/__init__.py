"""B300-native (sm_103a) per-tile heightmap build of LidarScout (HPG 2025).

Python binding of liblidarscout.so: the functions below only marshal torch CUDA
tensors into the C ABI of include/lidarscout.h; the work runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.

Points are dicts of CUDA tensors x, y, z (int32 centimetres) and r, g, b (uint16
stored as int16 or uint16 tensors), optionally with tile_offsets (int64, CSR by
tile).  A region is any object with x0_cm, y0_cm, tile_cm, tiles_x, tiles_y,
z_scale and z_offset attributes.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N

__all__ = ["bin_points", "bin_stats", "extract_samples", "extract_samples_into", "fill_sparse", "fill_interp",
           "update_tile", "render_framebuffer", "render_clear", "render_points", "render_heightmaps",
           "render_resolve", "PaperCNN", "PaperCNNFn", "cnn_inputs", "last_error",
           "release_workspace", "empty_bins", "BIN_KEYS", "Filler", "FillerFn", "filler_loss", "adamw_step",
           "learned_inputs", "learned_targets", "learned_finish", "fill_learned"]

BIN_KEYS = ("count", "zsum", "zmin", "zmax", "rsum", "gsum", "bsum")
_BIN_DTYPES = {"count": torch.int32, "zsum": torch.int64, "zmin": torch.int32, "zmax": torch.int32,
               "rsum": torch.int64, "gsum": torch.int64, "bsum": torch.int64}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return t


def _region(region):
    return N.LsRegion(int(region.x0_cm), int(region.y0_cm), int(region.tile_cm), int(region.tiles_x),
                      int(region.tiles_y), float(region.z_scale), float(region.z_offset))


def _points(p, need_offsets=False):
    for k in ("x", "y", "z"):
        _dev(p[k], k)
        assert p[k].dtype == torch.int32, f"{k} must be int32"
    for k in ("r", "g", "b"):
        _dev(p[k], k)
        assert p[k].element_size() == 2, f"{k} must be a 16-bit tensor"
    off = p.get("tile_offsets")
    if need_offsets and off is None:
        raise ValueError("tile_offsets (int64 CSR by tile) is required")
    if off is not None:
        _dev(off, "tile_offsets")
        assert off.dtype == torch.int64
    n = p["x"].numel()
    return N.LsPoints(_ptr(p["x"]), _ptr(p["y"]), _ptr(p["z"]), _ptr(p["r"]), _ptr(p["g"]),
                      _ptr(p["b"]), n, _ptr(off))


def empty_bins(n_tiles, cells, device="cuda"):
    """Uninitialised accumulator tensors [T, cells, cells] (uint64 sums in int64 storage,
    uint32 count in int32 storage)."""
    return {k: torch.empty((n_tiles, cells, cells), dtype=_BIN_DTYPES[k], device=device)
            for k in BIN_KEYS}


def _bins_struct(b, cells):
    return N.LsBins(cells, *[_ptr(_dev(b[k], k)) for k in BIN_KEYS])


def bin_points(points, region, levels=(640, 64), out=None, dropped=None, stream=None, accumulate=False):
    """Exact per-cell count / z-sum / z-min / z-max / RGB sums at one or two levels.

    accumulate=True adds the points into the bins and the dropped count given in `out`
    and `dropped` (points that arrive over several calls); both are then required.
    Returns (list of bin dicts, dropped tensor int64[1])."""
    if accumulate and (out is None or dropped is None):
        raise ValueError("accumulate=True needs the existing bins (out) and dropped counter")
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = points["x"].device
    if out is None:
        out = [empty_bins(T, c, dev) for c in levels]
    if dropped is None:
        dropped = torch.empty(1, dtype=torch.int64, device=dev)
    arr = (N.LsBins * len(levels))(*[_bins_struct(b, c) for b, c in zip(out, levels)])
    pts = _points(points)
    reg = _region(region)
    fn = "ls_bin_points_accumulate" if accumulate else "ls_bin_points"
    N.check(fn, getattr(N.lib(), fn)(ctypes.byref(pts), ctypes.byref(reg), arr, len(levels), _ptr(dropped),
                                     _stream(stream)))
    return out, dropped


def _shape_points(points):
    """An ls_points view for the shape table: only the count is read (host side)."""
    return N.LsPoints(None, None, None, None, None, None, int(points["x"].numel()), None)


def _level_structs(levels):
    return (N.LsBins * len(levels))(*[N.LsBins(int(c), None, None, None, None, None, None, None) for c in levels])


def bin_shape(points, levels=(640, 64)):
    """Launch shape {spans_per_cta, prefetch_batches} that binning these points uses."""
    out = N.LsBinShape()
    N.check("ls_bin_shape_get", N.lib().ls_bin_shape_get(ctypes.byref(_shape_points(points)), _level_structs(levels),
                                                        len(levels), ctypes.byref(out)))
    return {"spans_per_cta": out.spans_per_cta, "prefetch_batches": out.prefetch_batches}


def set_bin_shape(points, levels=(640, 64), shape=None):
    """Pins a binning launch shape (dict) for calls like this one; None removes it."""
    sh = None if shape is None else ctypes.byref(N.LsBinShape(int(shape["spans_per_cta"]),
                                                              int(shape["prefetch_batches"])))
    N.check("ls_bin_shape_set", N.lib().ls_bin_shape_set(ctypes.byref(_shape_points(points)), _level_structs(levels),
                                                        len(levels), sh))


def fill_shape(samples, n_out, res=64, radius_cm=12000, sigma_cm=4000.0):
    """Launch shape {split, ctas_per_sm} of a Gaussian fill call like this one."""
    out = N.LsFillShape()
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    N.check("ls_fill_shape_get", N.lib().ls_fill_shape_get(ctypes.byref(_shape_points(samples)), ctypes.byref(prm),
                                                          int(n_out), ctypes.byref(out)))
    return {"split": out.split, "ctas_per_sm": out.ctas_per_sm}


def set_fill_shape(samples, n_out, res=64, radius_cm=12000, sigma_cm=4000.0, shape=None):
    """Pins a fill launch shape (dict) for calls like this one; None removes it."""
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    sh = None if shape is None else ctypes.byref(N.LsFillShape(int(shape["split"]), int(shape["ctas_per_sm"])))
    N.check("ls_fill_shape_set", N.lib().ls_fill_shape_set(ctypes.byref(_shape_points(samples)), ctypes.byref(prm),
                                                          int(n_out), sh))


def tune_clear():
    """Forgets every tuned or pinned launch shape."""
    N.check("ls_tune_clear", N.lib().ls_tune_clear())


def tune_bin_points(points, region, levels=(640, 64), out=None, dropped=None, reps=5, stream=None):
    """Times every candidate binning shape on these points, keeps the fastest for calls
    like this one and leaves the bins computed.  Returns (shape dict, ms per call, out,
    dropped)."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = points["x"].device
    if out is None:
        out = [empty_bins(T, c, dev) for c in levels]
    if dropped is None:
        dropped = torch.empty(1, dtype=torch.int64, device=dev)
    arr = (N.LsBins * len(levels))(*[_bins_struct(b, c) for b, c in zip(out, levels)])
    best, ms = N.LsBinShape(), ctypes.c_float()
    N.check("ls_tune_bin_points", N.lib().ls_tune_bin_points(
        ctypes.byref(_points(points)), ctypes.byref(_region(region)), arr, len(levels), _ptr(dropped), int(reps),
        _stream(stream), ctypes.byref(best), ctypes.byref(ms)))
    return {"spans_per_cta": best.spans_per_cta, "prefetch_batches": best.prefetch_batches}, ms.value, out, dropped


def tune_fill_sparse(samples, region, tile_ids=None, res=64, radius_cm=12000, sigma_cm=4000.0, height=None,
                     rgb=None, reps=5, stream=None):
    """Times every valid fill shape on these samples, keeps the fastest for calls like
    this one and leaves the maps filled.  Returns (shape dict, ms per call, height, rgb)."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = samples["x"].device
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = T if tile_ids is None else tile_ids.numel()
    if height is None:
        height = torch.empty((n, res, res), dtype=torch.float32, device=dev)
    if rgb is None:
        rgb = torch.empty((n, res, res, 3), dtype=torch.uint8, device=dev)
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    best, ms = N.LsFillShape(), ctypes.c_float()
    N.check("ls_tune_fill_sparse", N.lib().ls_tune_fill_sparse(
        ctypes.byref(_points(samples, need_offsets=True)), ctypes.byref(_region(region)), ctypes.byref(prm),
        _ptr(tile_ids), n, _ptr(_dev(height, "height")), _ptr(_dev(rgb, "rgb")), int(reps), _stream(stream),
        ctypes.byref(best), ctypes.byref(ms)))
    return {"split": best.split, "ctas_per_sm": best.ctas_per_sm}, ms.value, height, rgb


def bin_stats(reset=True):
    """Binning diagnostics: late points, cross-CTA waits, waits that ran out, in-place
    flushes (cumulative since the last reset)."""
    out = (ctypes.c_uint64 * 4)()
    N.check("ls_bin_stats", N.lib().ls_bin_stats(out, int(reset)))
    return {"late_points": out[0], "waits": out[1], "wait_timeouts": out[2], "inplace_flushes": out[3]}


def extract_samples(points, chunk=50000, capacity=None, stream=None):
    """First point of every `chunk`-point chunk of every tile (needs tile_offsets).

    Returns a sample dict (x, y, z, r, g, b, tile_offsets) on the same device; the
    arrays are sized by the host-side capacity bound and trimmed after a sync."""
    pts = _points(points, need_offsets=True)
    off = points["tile_offsets"]
    T = off.numel() - 1
    n = points["x"].numel()
    if capacity is None:
        capacity = n // chunk + T
    dev = points["x"].device
    out = {k: torch.empty(max(capacity, 1), dtype=points[k].dtype, device=dev) for k in "xyzrgb"}
    soff = torch.empty(T + 1, dtype=torch.int64, device=dev)
    bufs = N.LsSampleBuffers(*[_ptr(out[k]) for k in "xyzrgb"])
    N.check("ls_extract_samples", N.lib().ls_extract_samples(ctypes.byref(pts), T, chunk, _ptr(soff),
                                                            ctypes.byref(bufs), capacity, _stream(stream)))
    total = int(soff[-1].item())
    out = {k: v[:min(total, capacity)] for k, v in out.items()}
    out["tile_offsets"] = soff
    return out


def extract_samples_into(points, samples, capacity, chunk=50000, stream=None):
    """Like extract_samples, into pre-allocated buffers (x, y, z, r, g, b of `capacity`
    entries and tile_offsets of T+1) without any host synchronisation, so the call can
    be captured in a CUDA graph.  The buffers past samples['tile_offsets'][-1] are
    unused."""
    pts = _points(points, need_offsets=True)
    T = points["tile_offsets"].numel() - 1
    bufs = N.LsSampleBuffers(*[_ptr(_dev(samples[k], k)) for k in "xyzrgb"])
    N.check("ls_extract_samples", N.lib().ls_extract_samples(
        ctypes.byref(pts), T, chunk, _ptr(_dev(samples["tile_offsets"], "tile_offsets")),
        ctypes.byref(bufs), capacity, _stream(stream)))
    return samples


def fill_sparse(samples, region, tile_ids=None, res=64, radius_cm=12000, sigma_cm=4000.0,
                height=None, rgb=None, stream=None):
    """Gaussian-weighted fill of res x res texels per requested tile.

    Returns (height float32 [n, res, res] metres, rgb uint8 [n, res, res, 3])."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = samples["x"].device
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = T if tile_ids is None else tile_ids.numel()
    if height is None:
        height = torch.empty((n, res, res), dtype=torch.float32, device=dev)
    if rgb is None:
        rgb = torch.empty((n, res, res, 3), dtype=torch.uint8, device=dev)
    pts = _points(samples, need_offsets=True)
    reg = _region(region)
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    N.check("ls_fill_sparse", N.lib().ls_fill_sparse(ctypes.byref(pts), ctypes.byref(reg), ctypes.byref(prm),
                                                    _ptr(tile_ids), n, _ptr(_dev(height, "height")),
                                                    _ptr(_dev(rgb, "rgb")), _stream(stream)))
    return height, rgb


INTERP_MAPS = ("nn_height", "nn_rgb", "lin_height", "lin_rgb", "inside")


def fill_interp(samples, region, tile_ids=None, res=96, pad_cm=16000, maps=INTERP_MAPS, tri_cap=0, out=None,
                stream=None):
    """Nearest-neighbour and Delaunay-linear maps of Alg. 1 on the padded patch of every
    requested tile (res x res texels of (tile + 2 pad) / res).

    Returns a dict with the requested maps: nn_height, lin_height float32 [n, res, res]
    (metres), nn_rgb, lin_rgb uint8 [n, res, res, 3], inside uint8 [n, res, res]; with
    tri_cap > 0 also triangles int32 [n, tri_cap, 3] (global sample indices, -1 - c for
    window corner c) and tri_count int32 [n].  `out` may hold pre-allocated tensors of those
    names (no allocation then, so the call can be captured in a CUDA graph)."""
    T = int(region.tiles_x) * int(region.tiles_y)
    dev = samples["x"].device
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = T if tile_ids is None else tile_ids.numel()
    shapes = {"nn_height": ((n, res, res), torch.float32), "lin_height": ((n, res, res), torch.float32),
              "nn_rgb": ((n, res, res, 3), torch.uint8), "lin_rgb": ((n, res, res, 3), torch.uint8),
              "inside": ((n, res, res), torch.uint8)}
    if tri_cap > 0:
        shapes["triangles"] = ((n, tri_cap, 3), torch.int32)
        shapes["tri_count"] = ((n,), torch.int32)
    res_maps = dict(out or {})
    for k, (shape, dt) in shapes.items():
        if k in res_maps or (k in INTERP_MAPS and k not in maps):
            continue
        res_maps[k] = torch.empty(shape, dtype=dt, device=dev)
    o = N.LsInterpOutputs(*[_ptr(_dev(res_maps[k], k)) if k in res_maps else None
                            for k in ("nn_height", "nn_rgb", "lin_height", "lin_rgb", "inside", "triangles",
                                      "tri_count")], int(tri_cap))
    pts = _points(samples, need_offsets=True)
    reg = _region(region)
    prm = N.LsInterpParams(res, pad_cm)
    N.check("ls_fill_interp", N.lib().ls_fill_interp(ctypes.byref(pts), ctypes.byref(reg), ctypes.byref(prm),
                                                    _ptr(tile_ids), n, ctypes.byref(o), _stream(stream)))
    return res_maps


def _camera(cam):
    """ls_camera from a dict with origin_cm (3 ints), view_proj (16 floats, row-major),
    width and height."""
    return N.LsCamera((N.I64 * 3)(*[int(v) for v in cam["origin_cm"]]),
                      (N.FLT * 16)(*[float(v) for v in cam["view_proj"]]), int(cam["width"]), int(cam["height"]))


def render_framebuffer(cam, device="cuda"):
    """An empty framebuffer (uint64 words stored in an int64 tensor [height, width])."""
    fb = torch.empty((int(cam["height"]), int(cam["width"])), dtype=torch.int64, device=device)
    return render_clear(fb)


def render_clear(fb, stream=None):
    N.check("ls_render_clear", N.lib().ls_render_clear(_ptr(_dev(fb, "fb")), fb.shape[1], fb.shape[0],
                                                      _stream(stream)))
    return fb


def render_points(points, cam, fb, stream=None):
    """Draw points (dict of x, y, z, r, g, b tensors) into the framebuffer."""
    pts = _points(points)
    c = _camera(cam)
    N.check("ls_render_points", N.lib().ls_render_points(ctypes.byref(pts), ctypes.byref(c),
                                                        _ptr(_dev(fb, "fb")), _stream(stream)))
    return fb


def render_heightmaps(height, rgb, region, cam, fb, tile_ids=None, stream=None):
    """Draw heightmaps (height float32 [n, res, res] metres, rgb uint8 [n, res, res, 3])
    of the tiles tile_ids (default 0..n-1) as triangle meshes."""
    n, res = height.shape[0], height.shape[1]
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=height.device, dtype=torch.int32).contiguous(), "tile_ids")
    c = _camera(cam)
    reg = _region(region)
    N.check("ls_render_heightmaps", N.lib().ls_render_heightmaps(
        _ptr(_dev(height, "height")), _ptr(_dev(rgb, "rgb")), _ptr(tile_ids), n, res, ctypes.byref(reg),
        ctypes.byref(c), _ptr(_dev(fb, "fb")), _stream(stream)))
    return fb


def render_resolve(fb, background=0, out=None, stream=None):
    """RGBA8 image uint8 [height, width, 4] of the framebuffer."""
    H, W = fb.shape
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=fb.device)
    N.check("ls_render_resolve", N.lib().ls_render_resolve(_ptr(_dev(fb, "fb")), W, H, int(background),
                                                          _ptr(_dev(out, "rgba")), _stream(stream)))
    return out


def update_tile(bins, region, tile_ids, height, rgb, stream=None):
    """Overwrite texels that hold full-resolution points with their mean (in place)."""
    cells = bins["count"].shape[-1]
    n = height.shape[0]
    if tile_ids is not None:
        tile_ids = _dev(tile_ids.to(device=height.device, dtype=torch.int32).contiguous(), "tile_ids")
    b = _bins_struct(bins, cells)
    reg = _region(region)
    N.check("ls_update_tile", N.lib().ls_update_tile(ctypes.byref(b), ctypes.byref(reg), _ptr(tile_ids), n,
                                                    _ptr(_dev(height, "height")), _ptr(_dev(rgb, "rgb")),
                                                    _stream(stream)))
    return height, rgb


def last_error():
    """Synchronise and return (then clear) the library's sticky device status."""
    return N.lib().ls_last_error()


def set_spin_limit(polls=0):
    """Polls before any bounded device wait gives up (0 restores the default)."""
    N.check("ls_set_spin_limit", N.lib().ls_set_spin_limit(int(polls)))


def probe_wait(flag, stream=None):
    """Run the binning's bounded row wait on a one-element int32 device tensor."""
    N.check("ls_probe_wait", N.lib().ls_probe_wait(_ptr(_dev(flag, "flag")), _stream(stream)))


def release_workspace():
    N.check("ls_release_workspace", N.lib().ls_release_workspace())


# ------------------------------------------------------------------------------------
# learned filler
# ------------------------------------------------------------------------------------

class Filler:
    """Native U-Net handle (ls_model) plus its flat fp32 parameter tensor.

    Layer order and layout as in include/lidarscout.h; ``params`` is a plain CUDA
    tensor that the caller may update (then call :meth:`load`)."""

    def __init__(self, widths=(32, 64, 128), res=64, max_batch=256, device="cuda", recompute=False):
        """recompute=True: activation recomputation per level (less device memory, one
        extra conv per level in backward, bit-identical results)."""
        self.widths, self.res, self.max_batch = tuple(widths), res, max_batch
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        w = (ctypes.c_int32 * len(widths))(*widths)
        N.check("ls_model_create_opts", N.lib().ls_model_create_opts(len(widths), w, res, max_batch,
                                                                    1 if recompute else 0, ctypes.byref(h)))
        self._h = h
        self.device_bytes = N.lib().ls_model_device_bytes(h)
        self.n_params = N.lib().ls_model_param_count(h)
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            N.lib().ls_model_destroy(h)
            self._h = None

    def layers(self):
        """[(cin, cout, k, w_offset, b_offset)] in parameter order."""
        out = []
        for i in range(N.lib().ls_model_layer_count(self._h)):
            a = [ctypes.c_int32() for _ in range(3)] + [ctypes.c_int64() for _ in range(2)]
            N.check("ls_model_layer_info", N.lib().ls_model_layer_info(self._h, i, *[ctypes.byref(v) for v in a]))
            out.append(tuple(v.value for v in a))
        return out

    def load(self, stream=None):
        N.check("ls_model_load", N.lib().ls_model_load(self._h, _ptr(self.params), _stream(stream)))

    def forward(self, x, stream=None):
        n = x.shape[0]
        y = torch.empty((n, self.res, self.res, 5), dtype=torch.float32, device=x.device)
        N.check("ls_filler_forward", N.lib().ls_filler_forward(self._h, _ptr(self.params), _ptr(_dev(x, "x")), n,
                                                              _ptr(y), _stream(stream)))
        return y

    def backward(self, dy, grads=None, stream=None):
        n = dy.shape[0]
        if grads is None:
            grads = torch.empty_like(self.params)
        N.check("ls_filler_backward", N.lib().ls_filler_backward(self._h, _ptr(self.params),
                                                                _ptr(_dev(dy.contiguous(), "dy")), n,
                                                                _ptr(grads), _stream(stream)))
        return grads


class FillerFn(torch.autograd.Function):
    """torch.autograd.Function whose forward and backward are the library's
    tensor-core kernels: y = filler(params; x), dL/dparams from dL/dy."""

    @staticmethod
    def forward(ctx, params, x, filler):
        ctx.filler = filler
        # the native backward reads the input of this forward (the first layer's weight
        # gradient): keep the tensor alive until then, or its memory may be reused
        ctx.x = x
        filler.load()
        return filler.forward(x)

    @staticmethod
    def backward(ctx, dy):
        return ctx.filler.backward(dy), None, None


class PaperCNN:
    """Native handle (ls_cnn) of the paper's network variant plus its flat fp32
    parameters: four encoders, two fully connected merge steps, height and texture
    decoders, skip concat with the inputs, final CNN, centre crop (see
    include/lidarscout.h).  Input: bf16 bits [n, res, res, 8] (cnn_inputs); output fp32
    [n, res/2, res/2, 5]."""

    def __init__(self, res=128, max_batch=256, training=True, device="cuda"):
        self.res, self.max_batch, self.training = res, max_batch, training
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        N.check("ls_cnn_create", N.lib().ls_cnn_create(res, max_batch, int(training), ctypes.byref(h)))
        self._h = h
        self.n_params = N.lib().ls_cnn_param_count(h)
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            N.lib().ls_cnn_destroy(h)
            self._h = None

    def layers(self):
        """[(kind, cin, cout, w_offset, b_offset)] in parameter order (kind 0: 3x3 conv,
        1: fully connected, 2: 1x1 head)."""
        out = []
        for i in range(N.lib().ls_cnn_layer_count(self._h)):
            a = [ctypes.c_int32() for _ in range(3)] + [ctypes.c_int64() for _ in range(2)]
            N.check("ls_cnn_layer_info", N.lib().ls_cnn_layer_info(self._h, i, *[ctypes.byref(v) for v in a]))
            out.append(tuple(v.value for v in a))
        return out

    def load(self, stream=None):
        N.check("ls_cnn_load", N.lib().ls_cnn_load(self._h, _ptr(self.params), _stream(stream)))

    def forward(self, x, stream=None):
        n = x.shape[0]
        y = torch.empty((n, self.res // 2, self.res // 2, 5), dtype=torch.float32, device=x.device)
        N.check("ls_cnn_forward", N.lib().ls_cnn_forward(self._h, _ptr(self.params), _ptr(_dev(x, "x")), n, _ptr(y),
                                                        _stream(stream)))
        return y

    def backward(self, dy, grads=None, stream=None):
        n = dy.shape[0]
        if grads is None:
            grads = torch.empty_like(self.params)
        N.check("ls_cnn_backward", N.lib().ls_cnn_backward(self._h, _ptr(self.params), _ptr(_dev(dy.contiguous(), "dy")),
                                                          n, _ptr(grads), _stream(stream)))
        return grads


class PaperCNNFn(torch.autograd.Function):
    """torch.autograd.Function over the library's kernels: y = cnn(params; x)."""

    @staticmethod
    def forward(ctx, params, x, cnn):
        ctx.cnn = cnn
        ctx.x = x  # read again by the native backward (see FillerFn)
        cnn.load()
        return cnn.forward(x)

    @staticmethod
    def backward(ctx, dy):
        return ctx.cnn.backward(dy), None, None


def cnn_inputs(maps, r_m=320.0, stream=None):
    """Network input of the paper's variant from ls_fill_interp maps (lin/nn height and
    rgb of n patches).  Returns (x bf16 bits int16 [n, res, res, 8], cz [n])."""
    lh = _dev(maps["lin_height"], "lin_height")
    n, res = lh.shape[0], lh.shape[1]
    x = torch.empty((n, res, res, 8), dtype=torch.int16, device=lh.device)
    cz = torch.empty(n, dtype=torch.float32, device=lh.device)
    N.check("ls_cnn_inputs", N.lib().ls_cnn_inputs(
        _ptr(lh), _ptr(_dev(maps["nn_height"], "nn_height")), _ptr(_dev(maps["lin_rgb"], "lin_rgb")),
        _ptr(_dev(maps["nn_rgb"], "nn_rgb")), n, res, float(r_m), _ptr(x), _ptr(cz), _stream(stream)))
    return x, cz


def filler_loss(y, base, target, mask, bound_weight=1.0, bound_excess=False, stream=None):
    """Masked, clipped MSE of Sec. 3.4 (+ bound term; bound_excess: its target is the
    excess of the learned height's error over the base fill's).  Returns (loss[4], dL/dy)."""
    n_px = mask.numel()
    sums = torch.empty(4, dtype=torch.float64, device=y.device)
    loss = torch.empty(4, dtype=torch.float32, device=y.device)
    dy = torch.empty_like(y)
    N.check("ls_filler_loss", N.lib().ls_filler_loss(_ptr(y), _ptr(base), _ptr(target), _ptr(mask), n_px,
                                                    float(bound_weight), int(bool(bound_excess)), _ptr(sums),
                                                    _ptr(loss), _ptr(dy), _stream(stream)))
    return loss, dy


def adamw_step(p, g, m, v, step, lr=1e-4, betas=(0.9, 0.999), eps=1e-5, weight_decay=1e-2, stream=None):
    N.check("ls_adamw_step", N.lib().ls_adamw_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr),
                                                  float(betas[0]), float(betas[1]), float(eps),
                                                  float(weight_decay), int(step), _stream(stream)))


def learned_inputs(samples, region, tile_ids, res=64, radius_cm=12000, sigma_cm=4000.0, stream=None):
    """Input raster of the filler for the given tiles.  Returns dict x (bf16 bits as
    int16 [n,res,res,8]), base [n,res,res,4], cz [n], fill_height, fill_rgb."""
    dev = samples["x"].device
    tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = tile_ids.numel()
    out = {"x": torch.empty((n, res, res, 8), dtype=torch.int16, device=dev),
           "base": torch.empty((n, res, res, 4), dtype=torch.float32, device=dev),
           "cz": torch.empty(n, dtype=torch.float32, device=dev),
           "fill_height": torch.empty((n, res, res), dtype=torch.float32, device=dev),
           "fill_rgb": torch.empty((n, res, res, 3), dtype=torch.uint8, device=dev)}
    aux = torch.empty(5 * n * res * res, dtype=torch.float32, device=dev)
    pts = _points(samples, need_offsets=True)
    reg = _region(region)
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    N.check("ls_learned_inputs", N.lib().ls_learned_inputs(
        ctypes.byref(pts), ctypes.byref(reg), ctypes.byref(prm), _ptr(tile_ids), n, _ptr(out["x"]),
        _ptr(out["base"]), _ptr(out["cz"]), _ptr(out["fill_height"]), _ptr(out["fill_rgb"]), _ptr(aux),
        _stream(stream)))
    return out


def learned_targets(bins, region, tile_ids, cz, stream=None):
    """Per-texel mean of the full-resolution points in patch space, and its mask."""
    cells = bins["count"].shape[-1]
    dev = cz.device
    tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n = tile_ids.numel()
    target = torch.empty((n, cells, cells, 4), dtype=torch.float32, device=dev)
    mask = torch.empty((n, cells, cells), dtype=torch.uint8, device=dev)
    b = _bins_struct(bins, cells)
    reg = _region(region)
    N.check("ls_learned_targets", N.lib().ls_learned_targets(ctypes.byref(b), ctypes.byref(reg), _ptr(tile_ids), n,
                                                            _ptr(cz), _ptr(target), _ptr(mask), _stream(stream)))
    return target, mask


def learned_finish(y, inputs, region, max_err_m=2.0, stream=None):
    n, res = y.shape[0], y.shape[1]
    height = torch.empty((n, res, res), dtype=torch.float32, device=y.device)
    rgb = torch.empty((n, res, res, 3), dtype=torch.uint8, device=y.device)
    bound = torch.empty(n, dtype=torch.float32, device=y.device)
    fb = torch.empty(n, dtype=torch.uint8, device=y.device)
    reg = _region(region)
    N.check("ls_learned_finish", N.lib().ls_learned_finish(
        _ptr(y), _ptr(inputs["base"]), _ptr(inputs["cz"]), n, res, ctypes.byref(reg), float(max_err_m),
        _ptr(inputs["fill_height"]), _ptr(inputs["fill_rgb"]), _ptr(height), _ptr(rgb), _ptr(bound), _ptr(fb),
        _stream(stream)))
    return height, rgb, bound, fb


def fill_learned(filler, samples, region, tile_ids, max_err_m=2.0, radius_cm=12000, sigma_cm=4000.0,
                 height=None, rgb=None, err_bound=None, used_fallback=None, scratch=None, stream=None):
    """Whole learned fill (input raster, network, finish with Gaussian fallback) of the
    given tiles in batches of the filler's max_batch."""
    dev = samples["x"].device
    tile_ids = _dev(tile_ids.to(device=dev, dtype=torch.int32).contiguous(), "tile_ids")
    n, res = tile_ids.numel(), filler.res
    if height is None:
        height = torch.empty((n, res, res), dtype=torch.float32, device=dev)
    if rgb is None:
        rgb = torch.empty((n, res, res, 3), dtype=torch.uint8, device=dev)
    if err_bound is None:
        err_bound = torch.empty(n, dtype=torch.float32, device=dev)
    if used_fallback is None:
        used_fallback = torch.empty(n, dtype=torch.uint8, device=dev)
    need = N.lib().ls_fill_learned_scratch_bytes(filler._h)
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    pts = _points(samples, need_offsets=True)
    reg = _region(region)
    prm = N.LsFillParams(res, radius_cm, sigma_cm)
    N.check("ls_fill_learned", N.lib().ls_fill_learned(
        filler._h, _ptr(filler.params), ctypes.byref(pts), ctypes.byref(reg), ctypes.byref(prm), _ptr(tile_ids),
        n, float(max_err_m), _ptr(height), _ptr(rgb), _ptr(err_bound), _ptr(used_fallback), _ptr(scratch),
        scratch.numel(), _stream(stream)))
    return height, rgb, err_bound, used_fallback
