"""Pins of the FP64 learned-filler oracle: conv against scipy, hand cases for pool,
upsample and the loss, finite differences for the whole backward pass (8x8
two-level and three-level instances), AdamW against torch.optim.AdamW (no GPU)."""
import numpy as np
import pytest
import scipy.signal

from oracle import unet as U


def test_param_count_of_32_64_128_net():
    # 3x3 convs 5-32-32 | 32-64-64 | 64-128-128 | 192-64-64 | 96-32-32, head 32->5
    assert U.param_count() == 472_261


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[n, :, :, i], w[o, :, :, i], mode="same")
                             for i in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_identity_kernel_returns_input():
    x = np.random.default_rng(1).standard_normal((1, 6, 6, 2))
    w = np.zeros((2, 3, 3, 2))
    w[0, 1, 1, 0] = w[1, 1, 1, 1] = 1.0
    np.testing.assert_array_equal(U.conv(x, w, np.zeros(2)), x)


def test_maxpool_and_backward_hand_case():
    x = np.array([[1., 5., 2., 2.], [5., 0., 2., 2.], [-1., -2., 0., 0.], [-3., -4., 0., 7.]])
    x = x.reshape(1, 4, 4, 1)
    np.testing.assert_array_equal(U.maxpool2(x)[0, :, :, 0], [[5., 2.], [-1., 7.]])
    d = U.maxpool2_backward(x, np.array([[10., 20.], [30., 40.]]).reshape(1, 2, 2, 1))[0, :, :, 0]
    # ties go to the first maximum in row-major window order
    np.testing.assert_array_equal(d, [[0., 10., 20., 0.], [0., 0., 0., 0.],
                                      [30., 0., 0., 0.], [0., 0., 0., 40.]])


def test_upsample_backward_sums_blocks():
    dy = np.arange(16.0).reshape(1, 4, 4, 1)
    np.testing.assert_array_equal(U.upsample2_backward(dy)[0, :, :, 0],
                                  [[0 + 1 + 4 + 5, 2 + 3 + 6 + 7], [8 + 9 + 12 + 13, 10 + 11 + 14 + 15]])


def test_loss_hand_case():
    y = np.zeros((1, 1, 2, 5))
    y[0, 0, 0] = [0.5, 0.1, 0.2, 0.3, 0.25]
    y[0, 0, 1] = [3.0, 0.0, 0.0, 0.0, 0.0]      # masked out
    base_h = np.array([[[0.0, 0.0]]])
    base_c = np.zeros((1, 1, 2, 3))
    t_h = np.array([[[2.0, 0.0]]])               # height error -1.5 -> squared 2.25 clipped to 1
    t_c = np.zeros((1, 1, 2, 3))
    mask = np.array([[[1, 0]]])
    loss, dy, parts = U.loss_and_grad(y, base_h, base_c, t_h, t_c, mask)
    assert parts["height"] == 1.0
    assert parts["color"] == pytest.approx((0.01 + 0.04 + 0.09) / 3)
    assert parts["bound"] == pytest.approx((0.25 - 1.5) ** 2)
    assert loss == pytest.approx(0.5 * (1.0 + 0.14 / 3) + 1.0 * 1.25 ** 2)
    assert dy[0, 0, 0, 0] == 0.0                 # clipped: no gradient
    assert dy[0, 0, 0, 1] == pytest.approx(0.5 * 2 * 0.1 / 3)
    assert dy[0, 0, 0, 4] == pytest.approx(2.0 * (0.25 - 1.5))
    assert (dy[0, 0, 1] == 0).all()


def test_loss_bound_excess_hand_case():
    """The excess target max(|e| - |e_base|, 0): the learned height's error over the
    base fill's error, zero where the learned height is the better one."""
    y = np.zeros((1, 1, 3, 5))
    y[0, 0, :, 0] = [0.3, -0.1, 0.0]             # residuals
    y[0, 0, :, 4] = [0.05, 0.2, 0.0]
    base_h = np.array([[[0.1, 0.5, -0.2]]])
    t_h = np.array([[[0.2, 0.2, 0.0]]])          # base errors -0.1, 0.3, -0.2
    z = np.zeros((1, 1, 3, 3))
    m = np.ones((1, 1, 3))
    # learned errors 0.2, 0.2, -0.2 -> excess 0.1, 0 (better than the base), 0
    _, dy, parts = U.loss_and_grad(y, base_h, z, t_h, z, m, bound_excess=True)
    tb = np.array([0.1, 0.0, 0.0])
    assert parts["bound"] == pytest.approx(((y[0, 0, :, 4] - tb) ** 2).mean())
    np.testing.assert_allclose(dy[0, 0, :, 4], 2.0 * (y[0, 0, :, 4] - tb) / 3.0, rtol=1e-12)
    # the absolute target on the same case: |e| = 0.2, 0.2, 0.2
    _, _, p_abs = U.loss_and_grad(y, base_h, z, t_h, z, m)
    assert p_abs["bound"] == pytest.approx(((y[0, 0, :, 4] - 0.2) ** 2).mean())


def _fd_check(widths, hw, n=2, seed=0, h=1e-6):
    layers = U.layer_table(widths)
    rng = np.random.default_rng(seed)
    params = U.init_params(seed, layers)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.standard_normal(params[k].shape) * 0.1
    x = rng.standard_normal((n, hw, hw, U.N_IN))
    gy = rng.standard_normal((n, hw, hw, U.N_OUT))

    def f(p):
        y, _ = U.forward(p, x, layers)
        return float((y * gy).sum())

    _, cache = U.forward(params, x, layers)
    g = U.backward(params, cache, gy, layers)
    worst = 0.0
    for k in params:
        flat = params[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            fp = f(params)
            flat[i] = old - h
            fm = f(params)
            flat[i] = old
            fd = (fp - fm) / (2 * h)
            an = g[k].reshape(-1)[i]
            worst = max(worst, abs(fd - an) / max(1.0, abs(fd), abs(an)))
    return worst


def test_backward_matches_finite_differences_8x8_two_level():
    assert _fd_check((4, 8), 8) < 1e-6


def test_backward_matches_finite_differences_three_level():
    assert _fd_check((4, 6, 8), 8, seed=3) < 1e-6


@pytest.mark.parametrize("excess", [False, True])
def test_loss_gradient_matches_finite_differences(excess):
    rng = np.random.default_rng(5)
    y = rng.standard_normal((2, 4, 4, 5)) * 0.3
    bh, bc = rng.standard_normal((2, 4, 4)) * 0.2, rng.random((2, 4, 4, 3))
    th, tc = rng.standard_normal((2, 4, 4)) * 0.2, rng.random((2, 4, 4, 3))
    m = rng.random((2, 4, 4)) > 0.3
    L = lambda yy: U.loss_and_grad(yy, bh, bc, th, tc, m, bound_excess=excess)  # noqa: E731
    _, dy, _ = L(y)

    def target(yy):
        t = np.abs(bh + yy[..., 0] - th)
        return np.maximum(t - np.abs(bh - th), 0.0) if excess else t

    h = 1e-7
    for _ in range(40):
        i = tuple(rng.integers(0, s) for s in y.shape)
        yp, ym = y.copy(), y.copy()
        yp[i] += h
        ym[i] -= h
        fd = (L(yp)[0] - L(ym)[0]) / (2 * h)
        if i[3] == 0:
            # the bound term's detached target also moves with y0: remove it
            db = lambda yy: ((yy[..., 4] - target(yy)) ** 2 * m).sum() / max(m.sum(), 1)  # noqa: E731
            fd -= (db(yp) - db(ym)) / (2 * h)
        assert fd == pytest.approx(dy[i], abs=1e-7)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-5, weight_decay=1e-2)
    for step in range(1, 6):
        g = rng.standard_normal(50)
        U.adamw_step(p, g, m, v, step, lr=1e-2)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_tile_inputs_hand_case():
    res, tile, cell = 8, 8000, 1000
    fill_h = np.full((res, res), 100.0)
    fill_h[3:5, 3:5] = 104.0                      # c_z = 104
    fill_c = np.full((res, res, 3), 128.0)
    nd2 = np.full((res, res), 0, np.int64)
    nd2[0, 0] = 3000 ** 2
    nd2[0, 1] = 99999 ** 2
    sx = np.array([2500, 2600, 99999]); sy = np.array([1500, 1700, 0])
    sz = np.array([10800, 20000, 0]); sr = np.array([65535, 0, 0])
    sg = np.array([0, 0, 0]); sb = np.array([0, 0, 0])
    x, bc, cz, r = U.tile_inputs(res, tile, cell, 0, 0, 0.01, 0.0, 2000,
                                 sx, sy, sz, sr, sg, sb, fill_h, fill_c, nd2)
    assert cz == 104.0 and r == 40.0
    # both samples fall in texel (1, 2); the lower index wins
    assert x[1, 2, 0] == pytest.approx((108.0 - 104.0) / 40.0)
    assert x[1, 2, 1] == pytest.approx(0.299)
    assert x[1, 2, 2] == 1.0 and x[..., 2].sum() == 1.0
    assert x[0, 0, 3] == 1.5 and x[0, 1, 3] == 2.0 and x[5, 5, 3] == 0.0
    assert x[0, 0, 4] == pytest.approx(-0.1) and x[4, 4, 4] == 0.0
    assert bc[0, 0, 0] == pytest.approx(128 * 256 / 65535)


def test_finish_hand_case():
    """Step a11 by hand: de-normalisation z'·r + c_z, colour clamp and half-up rounding,
    the bound as the RMS of the clamped error channel times r, and the fallback select
    on both sides of 2 m and on a NaN bound."""
    r = 320.0
    n, res = 5, 4
    y = np.zeros((n, res, res, 5))
    base_h = np.full((n, res, res), 0.5)
    base_c = np.full((n, res, res, 3), 0.25)
    cz = np.array([100.0, -20.0, 7.0, 0.0, 3.0])
    fill_h = np.full((n, res, res), -1.0)
    fill_rgb = np.full((n, res, res, 3), 9, np.uint8)
    y[..., 0] = 0.25                         # height = 0.75 * 320 + cz
    y[0, 0, 0, 1:4] = [0.25, 0.95, -0.5]     # colour 0.5 -> 128 (half up), 1.2 -> 255, -0.25 -> 0
    y[0, 0, 1, 1] = (63.5 - 1e-6) / 255.0 - 0.25   # just below a half level: rounds down to 63
    # tile 0: error channel all negative -> bound 0
    y[0, ..., 4] = -3.0
    # tile 1: a constant error channel gives bound = value * r; just under 2 m
    y[1, ..., 4] = (2.0 - 1e-9) / r
    # tile 2: just over 2 m
    y[2, ..., 4] = (2.0 + 1e-9) / r
    # tile 3: one NaN in the error channel -> NaN bound -> fallback
    y[3, 1, 2, 4] = np.nan
    # tile 4: half the texels at e and half negative: RMS = e / sqrt(2)
    y[4, :2, :, 4] = 2.0 * np.sqrt(2.0) / r * 0.999
    y[4, 2:, :, 4] = -1.0
    h, c, bound, used = U.finish(y, base_h, base_c, cz, r, fill_h, fill_rgb, 2.0)
    assert bound[0] == 0.0
    assert bound[1] == pytest.approx(2.0 - 1e-9, abs=1e-12) and used[1] == 0
    assert bound[2] == pytest.approx(2.0 + 1e-9, abs=1e-12) and used[2] == 1
    assert np.isnan(bound[3]) and used[3] == 1
    assert bound[4] == pytest.approx(2.0 * 0.999) and used[4] == 0
    assert list(used) == [0, 0, 1, 1, 0]
    for o in (0, 1, 4):
        np.testing.assert_allclose(h[o], 0.75 * r + cz[o], rtol=0, atol=1e-12)
    for o in (2, 3):
        assert (h[o] == -1.0).all() and (c[o] == 9).all()
    assert list(c[0, 0, 0]) == [128, 255, 0]
    assert c[0, 0, 1, 0] == 63
    assert (c[1] == 64).all()            # 0.25 * 255 = 63.75 -> 64
