"""GPU parity of the tcgen05 3x3 convolution against the FP64 oracle conv evaluated on
the same bf16-rounded operands.  Tolerance: the output is rounded to bf16 (relative
2^-9) after an FP32 accumulation of up to 1728 products, so
|gpu - ref| <= 2^-7 |ref| + 2^-9 max|ref| is required elementwise."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


def bf16_bits(a):
    """Round float32 to bfloat16 (nearest even); returns uint16 bit patterns."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r


def bf16_to_f64(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def lib():
    from paper_2509_20198_b300 import build, _native
    build.build_library()
    return _native


def _run_conv(N, x_bits, w, b, mask_bits, relu, shape, flip=False):
    import ctypes
    import torch
    n, h, wd, cin, cout = shape
    L = N.lib()
    pk = torch.empty(L.ls_conv3x3_packed_elems(cin, cout), dtype=torch.int16, device="cuda")
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    N.check("pack", L.ls_conv3x3_pack(ctypes.c_void_p(wt.data_ptr()), cin, cout, int(flip),
                                      ctypes.c_void_p(pk.data_ptr()), None))
    xt = torch.from_numpy(x_bits.view(np.int16)).cuda()
    bt = None if b is None else torch.from_numpy(np.asarray(b, np.float32)).cuda()
    mt = None if mask_bits is None else torch.from_numpy(mask_bits.view(np.int16)).cuda()
    y = torch.empty((n, h, wd, cout), dtype=torch.int16, device="cuda")
    sh = N.LsConvShape(n, h, wd, cin, cout)
    N.check("conv", L.ls_conv3x3_forward(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(pk.data_ptr()),
                                         None if bt is None else ctypes.c_void_p(bt.data_ptr()),
                                         None if mt is None else ctypes.c_void_p(mt.data_ptr()),
                                         int(relu), ctypes.byref(sh), ctypes.c_void_p(y.data_ptr()), None))
    torch.cuda.synchronize()
    assert L.ls_last_error() == 0
    return bf16_to_f64(y.cpu().numpy().view(np.uint16))


def _close(g, r):
    tol = 2.0 ** -7 * np.abs(r) + 2.0 ** -9 * np.abs(r).max()
    bad = np.abs(g - r) > tol
    assert not bad.any(), f"{bad.sum()} of {bad.size} outside tolerance, max err {np.abs(g - r).max():.3e}"


SHAPES = [
    (2, 64, 64, 8, 32),     # first layer (5 channels padded to 8)
    (2, 32, 32, 32, 64),
    (1, 16, 16, 64, 128),
    (2, 32, 32, 192, 64),   # decoder concat width
    (1, 64, 64, 96, 32),
    (16, 4, 4, 8, 16),      # several whole images per 128-pixel tile
    (2, 16, 16, 128, 256),
    (2, 64, 64, 16, 32),    # 16-channel blocks (32-byte swizzle)
    (1, 128, 128, 48, 32),  # the skip concat: 16-channel blocks, 128-wide rows
    (2, 64, 64, 64, 32),    # halo form, 64-channel blocks (128-byte swizzle), two pipelines
    (2, 64, 64, 32, 64),    # halo form, four pipelines of 64 accumulator columns
    (1, 128, 128, 8, 16),   # halo form, 8-channel input on 130-slot rows
    (3, 20, 32, 32, 32),    # halo form, 34-slot rows, images padded to whole tiles
    (1, 37, 64, 16, 32),    # halo form, odd height: junk rows in the last tile
    (3, 20, 32, 160, 48),   # streamed weights: three pipelines share each 3-tile box
    (2, 64, 64, 256, 64),   # streamed weights, four pipelines, tiles past the image skipped
    (1, 37, 64, 192, 32),   # streamed weights, odd height
    (1, 64, 64, 32, 128),   # halo form, two pipelines of 128 accumulator columns
    (2, 32, 32, 256, 128),  # streamed weights, two pipelines sharing 2-tile boxes
]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_bias_relu(lib, shape):
    n, h, w, cin, cout = shape
    rng = np.random.default_rng(cin * 1000 + cout)
    x = bf16_bits(rng.standard_normal((n, h, w, cin)).astype(np.float32))
    wt = (rng.standard_normal((cout, 3, 3, cin)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    b = (rng.standard_normal(cout) * 0.1).astype(np.float32)
    g = _run_conv(lib, x, wt, b, None, True, shape)
    wq = bf16_to_f64(bf16_bits(wt))
    ref = U.relu(U.conv(bf16_to_f64(x), wq, b.astype(np.float64)))
    _close(g, ref)


@pytest.mark.parametrize("shape", [(2, 32, 32, 64, 32), (2, 64, 64, 32, 32)])
def test_mask_epilogue_and_no_bias(lib, shape):
    n, h, w, cin, cout = shape
    rng = np.random.default_rng(3)
    x = bf16_bits(rng.standard_normal((n, h, w, cin)).astype(np.float32))
    wt = (rng.standard_normal((cout, 3, 3, cin)) * 0.05).astype(np.float32)
    mask_f = rng.standard_normal((n, h, w, cout)).astype(np.float32)
    mask_f[mask_f < -1.0] = 0.0
    mask = bf16_bits(mask_f)
    g = _run_conv(lib, x, wt, None, mask, False, shape)
    ref = U.conv(bf16_to_f64(x), bf16_to_f64(bf16_bits(wt)), np.zeros(cout)) * (bf16_to_f64(mask) > 0)
    _close(g, ref)


@pytest.mark.parametrize("shape", [(2, 32, 32, 64, 32), (1, 64, 64, 32, 96)])
def test_input_gradient_via_flipped_weights(lib, shape):
    """dX of a conv (c_in -> c_out) = conv(dY, W') with the transposed, flipped pack."""
    n, h, w, ci, co = shape          # original layer: ci -> co
    rng = np.random.default_rng(ci + co)
    dy = bf16_bits(rng.standard_normal((n, h, w, co)).astype(np.float32))
    wt = (rng.standard_normal((co, 3, 3, ci)) * 0.05).astype(np.float32)
    g = _run_conv(lib, dy, wt, None, None, False, (n, h, w, co, ci), flip=True)
    x_dummy = np.zeros((n, h, w, ci))
    dx, _, _ = U.conv_backward(x_dummy, bf16_to_f64(bf16_bits(wt)), bf16_to_f64(dy))
    _close(g, dx)


WGRAD_SHAPES = [
    (16, 4, 4, 16, 16), (2, 128, 128, 8, 16), (1, 128, 128, 48, 32),
    (2, 64, 64, 16, 48),      # per-tap form (input channels not in blocks of 32, or narrow images)
    (2, 64, 64, 8, 32),       # eight-channel halo form: dZ rows as A, input views as B
    (1, 9, 16, 8, 32),        # eight-channel halo form, 16-wide rows, ragged height
    (2, 7, 32, 8, 64),        # eight-channel halo form, two M tiles (C_out = 64)
    (1, 4, 128, 8, 64),       # eight-channel halo form, 128-wide rows
    (2, 32, 32, 32, 64),      # halo form: one block, 64 accumulator columns per tile
    (1, 16, 16, 64, 128),     # halo form, 16-wide rows, two CTA groups of one block
    (2, 32, 32, 192, 64),     # halo form, three CTA groups of two blocks (decoder concat)
    (1, 64, 64, 96, 32),      # halo form, nine M tiles and issuers (three blocks)
    (2, 64, 64, 32, 32), (2, 32, 32, 64, 64), (1, 16, 16, 128, 128),
    (3, 22, 32, 32, 32),      # halo form, height not a multiple of the 4-row chunk
    (1, 37, 64, 32, 32),      # halo form, odd height
    (1, 8, 128, 32, 32),      # halo form, 128-wide rows (one row per chunk)
    (2, 5, 16, 192, 64),      # halo form, fewer chunks than slices
    (1, 9, 32, 32, 96),       # halo form, three 32-channel dZ blocks
    (1, 6, 64, 128, 32),      # halo form, four channel blocks in one CTA
]


@pytest.mark.parametrize("shape", WGRAD_SHAPES)
def test_weight_gradient_matches_oracle(lib, shape):
    """dW, db of the tcgen05 weight-gradient GEMM against the FP64 oracle on the same
    bf16 operands.  The products are exact in FP32; the sums over n*h*w pixels are FP32,
    so each element is within 2^-12 of the sum of the magnitudes of its products (and the
    whole gradient within 1e-4 relative L2)."""
    import ctypes
    import torch
    n, h, w, cin, cout = shape
    rng = np.random.default_rng(cin * 7 + cout)
    x = bf16_bits(np.maximum(rng.standard_normal((n, h, w, cin)), 0).astype(np.float32))
    dz = bf16_bits((rng.standard_normal((n, h, w, cout)) * (rng.random((n, h, w, cout)) > 0.3)).astype(np.float32))
    xt = torch.from_numpy(x.view(np.int16)).cuda()
    dt = torch.from_numpy(dz.view(np.int16)).cuda()
    dw = torch.zeros(9 * cin * cout, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    L = lib.lib()
    sh = lib.LsConvShape(n, h, w, cin, cout)
    lib.check("wgrad", L.ls_conv3x3_wgrad(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(dt.data_ptr()),
                                          ctypes.byref(sh), ctypes.c_void_p(dw.data_ptr()),
                                          ctypes.c_void_p(db.data_ptr()), None))
    torch.cuda.synchronize()
    assert L.ls_last_error() == 0
    _, gw, gb = U.conv_backward(bf16_to_f64(x), np.zeros((cout, 3, 3, cin)), bf16_to_f64(dz))
    g = dw.cpu().numpy().astype(np.float64).reshape(3, 3, cin, cout).transpose(3, 0, 1, 2)
    rel = np.linalg.norm(g - gw) / np.linalg.norm(gw)
    assert rel < 1e-4, rel
    _, aw, _ = U.conv_backward(np.abs(bf16_to_f64(x)), np.zeros((cout, 3, 3, cin)), np.abs(bf16_to_f64(dz)))
    bad = np.abs(g - gw) > 2.0 ** -12 * aw + 1e-30
    assert not bad.any(), f"{bad.sum()} of {bad.size} elements outside 2^-12 of the magnitude sum"
    np.testing.assert_allclose(db.cpu().numpy(), gb, rtol=1e-4, atol=1e-3)
