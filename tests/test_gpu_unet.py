"""GPU parity of the learned filler: tensor-core forward and backward against the
FP64 oracle on the same bf16-rounded weights and inputs, against torch autograd as an
independent reference gradient, plus loss, AdamW, input raster, targets and the
learned fill with its Gaussian fallback.

Tolerances (derived from the arithmetic): every conv output and every activation
gradient is stored in bf16 (2^-8 relative per ulp, 2^-9 when rounded to nearest).
A parameter gradient dW = X^T dZ depends on the 11 stored conv outputs of the forward
pass (X and the ReLU masks that shape dZ) and on one stored gradient per layer
between it and the loss (its depth, 0 for the head).  Against the oracle that rounds
at the same places (bf16 storage, FP64 arithmetic) a stored value differs by at most
one ulp, where fp32 and FP64 accumulation put it on different sides of a rounding
boundary, so the relative L2 error is below (11 + depth)·2^-8 and the cosine above
1 - bar^2/2.  Against pure FP64 (the oracle and torch autograd), bf16 rounding moves
near-zero pre-activations across the ReLU threshold, a discrete change that no ulp
count bounds: with random signs only the direction is checked (cosine > 0.95); with
every ReLU active (non-negative inputs and weights, positive biases) there are no
such flips, and the relative L2 error of every layer whose output gradient does not
pass back through a max pool (a near-tie there can route it to another texel) is
below (11 + depth)·2^-9.  The forward output
(11 stored convs) is compared by relative L2 below 3e-2 (FP64) and 2e-2 (bf16
storage).  The loss and AdamW run in fp32 and match to 1e-5."""
import numpy as np
import pytest

import oracle
import synth
from oracle import unet as U
from tests.helpers import to_device
from tests.test_gpu_conv import bf16_bits, bf16_to_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    return lsb


def _flat(params, layers):
    return np.concatenate([np.concatenate([params[n + ".w"].ravel(), params[n + ".b"].ravel()])
                           for n, *_ in layers]).astype(np.float32)


def _setup(lsb, widths, n, seed):
    import torch
    layers = U.layer_table(widths)
    rng = np.random.default_rng(seed)
    params = U.init_params(seed, layers)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.standard_normal(params[k].shape) * 0.05
    f = lsb.Filler(widths=widths, res=64, max_batch=max(n, 2))
    assert f.n_params == U.param_count(layers)
    flat = _flat(params, layers)
    f.params.copy_(torch.from_numpy(flat))
    f.load()
    x5 = rng.standard_normal((n, 64, 64, 5)).astype(np.float32) * 0.5
    x5[..., 2] = (rng.random((n, 64, 64)) < 0.02)
    xb = bf16_bits(np.concatenate([x5, np.zeros((n, 64, 64, 3), np.float32)], axis=3))
    # oracle operands: bf16-rounded 3x3 weights (the tensor-core operands), fp32 head
    q = {}
    for name, ci, co, k in layers:
        w = params[name + ".w"].astype(np.float32)
        q[name + ".w"] = bf16_to_f64(bf16_bits(w)) if k == 3 else w.astype(np.float64)
        q[name + ".b"] = params[name + ".b"].astype(np.float32).astype(np.float64)
    xo = bf16_to_f64(xb)[..., :5]
    return f, layers, params, q, xb, xo


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _cos(a, b):
    return float((a * b).sum() / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("widths,n", [((32, 64, 128), 2), ((32, 64), 3)])
def test_forward_matches_oracle(lsb, widths, n):
    import torch
    f, layers, params, q, xb, xo = _setup(lsb, widths, n, 1)
    y = f.forward(torch.from_numpy(xb.view(np.int16)).cuda()).cpu().numpy().astype(np.float64)
    assert lsb.last_error() == 0
    yr, _ = U.forward(q, xo, layers)
    assert _rel(y, yr) < 3e-2 and _cos(y.ravel(), yr.ravel()) > 0.999
    rnd = lambda a: bf16_to_f64(bf16_bits(a.astype(np.float32)))  # noqa: E731
    yb, _ = U.forward(q, xo, layers, store=rnd)
    print("forward rel err vs FP64 oracle", _rel(y, yr), "vs bf16-storage oracle", _rel(y, yb))
    assert _rel(y, yb) < 2e-2


def test_backward_matches_oracle_and_torch(lsb):
    import torch
    widths, n = (32, 64, 128), 2
    f, layers, params, q, xb, xo = _setup(lsb, widths, n, 2)
    xt = torch.from_numpy(xb.view(np.int16)).cuda()
    y = f.forward(xt)
    rng = np.random.default_rng(5)
    dy = rng.standard_normal(y.shape).astype(np.float32) * 1e-3
    g = f.backward(torch.from_numpy(dy).cuda()).cpu().numpy().astype(np.float64)
    assert lsb.last_error() == 0
    yr, cache = U.forward(q, xo, layers)
    gr = U.backward(q, cache, dy.astype(np.float64), layers)
    # the oracle with values rounded to bf16 wherever the kernels store them (its
    # arithmetic stays FP64): isolates the backward logic from storage precision
    rnd = lambda a: bf16_to_f64(bf16_bits(a.astype(np.float32)))  # noqa: E731
    _, cache_b = U.forward(q, xo, layers, store=rnd)
    gb16 = U.backward(q, cache_b, dy.astype(np.float64), layers, store=rnd)
    # torch autograd (fp64, CPU) on the same operands: an independent reference gradient
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in q.items()}
    h = torch.tensor(xo).permute(0, 3, 1, 2)
    skips = []
    L = len(widths)
    for l in range(1, L + 1):
        if l > 1:
            h = torch.nn.functional.max_pool2d(h, 2)
        for s in "ab":
            w = tp[f"e{l}{s}.w"].permute(0, 3, 1, 2)
            h = torch.relu(torch.nn.functional.conv2d(h, w, tp[f"e{l}{s}.b"], padding=1))
        skips.append(h)
    for l in range(L - 1, 0, -1):
        h = torch.cat([torch.nn.functional.interpolate(h, scale_factor=2, mode="nearest"), skips[l - 1]], 1)
        for s in "ab":
            w = tp[f"d{l}{s}.w"].permute(0, 3, 1, 2)
            h = torch.relu(torch.nn.functional.conv2d(h, w, tp[f"d{l}{s}.b"], padding=1))
    yt = torch.nn.functional.conv2d(h, tp["head.w"].permute(0, 3, 1, 2), tp["head.b"]).permute(0, 2, 3, 1)
    (yt * torch.tensor(dy, dtype=torch.float64)).sum().backward()
    off = 0
    errs = {}
    for name, ci, co, k in layers:
        nw = co * k * k * ci
        gw, gb = g[off:off + nw].reshape(co, k, k, ci), g[off + nw:off + nw + co]
        off += nw + co
        for ref, msg in ((gr, "oracle"), ({kk: tp[kk].grad.numpy() for kk in tp}, "torch"),
                         (gb16, "oracle-bf16-storage")):
            errs[(name, msg)] = (_rel(gw, ref[name + ".w"]), _cos(gw.ravel(), ref[name + ".w"].ravel()),
                                 _rel(gb, ref[name + ".b"]))
    print({k: tuple(round(float(x), 4) for x in v) for k, v in errs.items()})
    depth = {name: len(layers) - 1 - i for i, (name, _, _, _) in enumerate(layers)}
    n_stored = len(layers) - 1                     # conv outputs stored in bf16
    for (name, msg), (rw, cw, rb) in errs.items():
        if msg == "oracle-bf16-storage":
            bar = (n_stored + depth[name]) * 2.0 ** -8
            assert rw < bar and rb < bar, (name, msg, rw, rb, bar)
            assert cw > 1.0 - bar * bar / 2, (name, msg, cw, bar)
            continue
        assert cw > 0.95, (name, msg, cw)          # direction only: ReLU flips (see above)


def test_backward_with_every_relu_active_matches_fp64(lsb):
    """Non-negative inputs and weights and positive biases keep every pre-activation
    well above zero, so no ReLU branch flips.  For the layers whose output gradient
    does not pass back through a max pool (bottom level, decoder, head) bf16 rounding
    is then the only error: within (11 + depth)·2^-9 of FP64 in relative L2.  The
    encoder layers above a pool (a near-tie in a window may route its gradient to the
    other texel) are checked for direction (cosine > 0.95)."""
    import torch
    widths, n = (32, 64, 128), 2
    layers = U.layer_table(widths)
    rng = np.random.default_rng(12)
    params = U.init_params(12, layers)
    for name, ci, co, k in layers:
        # |w| with mean 1.25 / (ci k k): activations stay of the order of the input
        params[name + ".w"] = np.abs(rng.standard_normal((co, k, k, ci))) * (1.25 / (ci * k * k))
        params[name + ".b"] = 0.05 + 0.05 * rng.random(co)
    f = lsb.Filler(widths=widths, res=64, max_batch=n)
    f.params.copy_(torch.from_numpy(_flat(params, layers)))
    f.load()
    q = {}
    for name, ci, co, k in layers:
        w = params[name + ".w"].astype(np.float32)
        q[name + ".w"] = bf16_to_f64(bf16_bits(w)) if k == 3 else w.astype(np.float64)
        q[name + ".b"] = params[name + ".b"].astype(np.float32).astype(np.float64)
    x5 = rng.random((n, 64, 64, 5)).astype(np.float32)
    xb = bf16_bits(np.concatenate([x5, np.zeros((n, 64, 64, 3), np.float32)], axis=3))
    xo = bf16_to_f64(xb)[..., :5]
    y = f.forward(torch.from_numpy(xb.view(np.int16)).cuda())
    dy = rng.random(tuple(y.shape)).astype(np.float32) * 1e-3
    g = f.backward(torch.from_numpy(dy).cuda()).cpu().numpy().astype(np.float64)
    assert lsb.last_error() == 0
    yr, cache = U.forward(q, xo, layers)
    for name in [nm for nm, *_ in layers if nm != "head"]:
        assert (cache[name] > 0).all(), name           # every ReLU active in the oracle
    gr = U.backward(q, cache, dy.astype(np.float64), layers)
    depth = {name: len(layers) - 1 - i for i, (name, _, _, _) in enumerate(layers)}
    above_pool = {f"e{l}{s}" for l in range(1, len(widths)) for s in "ab"}
    off = 0
    seen = {}
    for name, ci, co, k in layers:
        nw = co * k * k * ci
        gw, gb = g[off:off + nw].reshape(co, k, k, ci), g[off + nw:off + nw + co]
        off += nw + co
        bar = (len(layers) - 1 + depth[name]) * 2.0 ** -9
        rw, rb = _rel(gw, gr[name + ".w"]), _rel(gb, gr[name + ".b"])
        seen[name] = (round(rw, 5), round(rb, 5), round(bar, 4))
        if name in above_pool:
            assert _cos(gw.ravel(), gr[name + ".w"].ravel()) > 0.95, (name, rw)
            continue
        assert rw < bar and rb < bar, (name, rw, rb, bar)
    print(seen)


@pytest.mark.parametrize("widths", [(32, 64, 128), (16, 32)])
def test_recompute_per_level_is_bit_identical_and_smaller(lsb, widths):
    """Activation recomputation per level: the outputs and every gradient equal those
    of the model that keeps all activations, bit for bit, in less device memory."""
    import torch
    n = 8
    f, layers, params, q, xb, xo = _setup(lsb, widths, n, seed=5)
    g = lsb.Filler(widths=widths, res=64, max_batch=max(n, 2), recompute=True)
    g.params.copy_(f.params)
    g.load()
    assert g.device_bytes < f.device_bytes
    x = torch.from_numpy(xb.view(np.int16)).cuda()
    dy = torch.from_numpy(np.random.default_rng(6).standard_normal((n, 64, 64, 5)).astype(np.float32)).cuda()
    y1, y2 = f.forward(x), g.forward(x)
    g1, g2 = f.backward(dy), g.backward(dy)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    assert torch.equal(y1, y2)
    assert torch.equal(g1, g2)
    assert float(g1.abs().sum()) > 0


def test_loss_and_adamw_match_oracle(lsb):
    import torch
    rng = np.random.default_rng(7)
    n = 3
    y = (rng.standard_normal((n, 64, 64, 5)) * 0.3).astype(np.float32)
    base = rng.standard_normal((n, 64, 64, 4)).astype(np.float32) * 0.2
    tgt = rng.standard_normal((n, 64, 64, 4)).astype(np.float32) * 0.2
    tgt[0, :4, :4, 0] += 3.0     # clipped squared errors
    mask = (rng.random((n, 64, 64)) > 0.2).astype(np.uint8)
    T = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    for excess in (False, True):
        loss, dy = lsb.filler_loss(T(y), T(base), T(tgt), T(mask), bound_excess=excess)
        lr_, dyr, parts = U.loss_and_grad(y.astype(np.float64), base[..., 0].astype(np.float64),
                                          base[..., 1:].astype(np.float64), tgt[..., 0].astype(np.float64),
                                          tgt[..., 1:].astype(np.float64), mask, bound_excess=excess)
        l4 = loss.cpu().numpy()
        assert l4[0] == pytest.approx(lr_, rel=1e-5)
        assert l4[1] == pytest.approx(parts["height"], rel=1e-5)
        assert l4[3] == pytest.approx(parts["bound"], rel=1e-5)
        # the bound gradient 2 (y4 - b)/n cancels in fp32 where y4 ~ b (b a difference
        # of fp32 terms): absolute tolerance of a few fp32 ulps of |y4| / n
        np.testing.assert_allclose(dy.cpu().numpy(), dyr, rtol=1e-5, atol=4e-6 / mask.sum())
    # AdamW
    p = rng.standard_normal(1000).astype(np.float32)
    pg, pm, pv = T(p.copy()), T(np.zeros(1000, np.float32)), T(np.zeros(1000, np.float32))
    po, mo, vo = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in range(1, 4):
        gr = rng.standard_normal(1000).astype(np.float32)
        lsb.adamw_step(pg, T(gr), pm, pv, step, lr=1e-3)
        U.adamw_step(po, gr.astype(np.float64), mo, vo, step, lr=1e-3)
    np.testing.assert_allclose(pg.cpu().numpy(), po, rtol=1e-5, atol=1e-6)


def test_input_raster_and_targets_match_oracle(lsb):
    import torch
    region = synth.Region(tiles_x=4, tiles_y=3)
    counts = synth.uniform_counts(12, 4.0)
    counts[5] = 2_000_000
    s = synth.region_samples(21, region, counts)
    tiles = np.array([5, 0, 11], np.int64)
    inp = lsb.learned_inputs(to_device(s), region, torch.as_tensor(tiles))
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    ref = oracle.fill_sparse(s, region, tile_ids=tiles)
    x = bf16_to_f64(inp["x"].cpu().numpy().view(np.uint16))
    for o, t in enumerate(tiles):
        tx, ty = t % region.tiles_x, t // region.tiles_x
        a, b = s["tile_offsets"][t], s["tile_offsets"][t + 1]
        xr, bc, cz, r = U.tile_inputs(64, 64000, 1000, region.x0_cm + tx * 64000, region.y0_cm + ty * 64000,
                                      0.01, 0.0, 12000, s["x"][a:b], s["y"][a:b], s["z"][a:b], s["r"][a:b],
                                      s["g"][a:b], s["b"][a:b], ref["height"][o], ref["rgbf"][o],
                                      ref["nearest_d2"][o])
        assert inp["cz"][o].item() == pytest.approx(cz, abs=1e-3)
        # bf16 channels: relative 2^-8 plus the fp32 fill error (1e-3 m / 320 m)
        np.testing.assert_allclose(x[o, ..., :5], xr, rtol=2 ** -8, atol=2e-5)
        assert (x[o, ..., 5:] == 0).all()
        np.testing.assert_allclose(inp["base"][o, ..., 1:].cpu().numpy(), bc, atol=1e-4)
    # targets from the full-resolution bins of tile 5
    pts = synth.region_points(21, region, np.where(np.arange(12) == 5, counts, 0))
    (b64,), _ = lsb.bin_points(to_device(pts), region, levels=(64,))
    tgt, mask = lsb.learned_targets(b64, region, torch.as_tensor(tiles[:1]), inp["cz"][:1])
    ob = oracle.bin_points(pts, region, 64)
    cnt = ob["count"][5]
    m = cnt > 0
    assert (mask[0].cpu().numpy().astype(bool) == m).all()
    zm = ob["zsum"][5][m] / cnt[m] * 0.01
    np.testing.assert_allclose(tgt[0, ..., 0].cpu().numpy()[m], (zm - inp["cz"][0].item()) / 320.0, atol=1e-6)
    np.testing.assert_allclose(tgt[0, ..., 1].cpu().numpy()[m], ob["rsum"][5][m] / cnt[m] / 65535.0, atol=1e-6)


def test_fill_learned_fallback_and_finish(lsb):
    import torch
    region = synth.Region(tiles_x=3, tiles_y=3)
    counts = synth.uniform_counts(9, 4.0)
    s = to_device(synth.region_samples(22, region, counts))
    f = lsb.Filler(max_batch=4)
    f.params.normal_(0, 0.02)
    f.load()
    tiles = torch.arange(9, dtype=torch.int32)
    gh, gc = lsb.fill_sparse(s, region)
    h0, c0, b0, fb0 = lsb.fill_learned(f, s, region, tiles, max_err_m=-1.0)     # everything falls back
    assert (fb0 == 1).all() and torch.equal(h0, gh) and torch.equal(c0, gc)
    h1, c1, b1, fb1 = lsb.fill_learned(f, s, region, tiles, max_err_m=1e30)     # nothing falls back
    assert (fb1 == 0).all()
    inp = lsb.learned_inputs(s, region, tiles)
    y = torch.cat([f.forward(inp["x"][a:a + 4].contiguous()) for a in range(0, 9, 4)])
    h2, c2, b2, _ = lsb.learned_finish(y, inp, region, max_err_m=1e30)
    assert torch.allclose(h1, h2) and torch.equal(c1, c2)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0


def test_learned_finish_matches_oracle(lsb):
    """Step a11 alone: ls_learned_finish on seeded network outputs against the FP64
    oracle's finish.  Heights: three fp32 roundings of (base + y0)·r + c_z, so within
    2^-22·(|base + y0|·r + |c_z|) + 1e-7 m.  Colours: exact away from a rounding
    boundary (the fp32 sum base + y carries 2^-24 relative error, far below 1e-4 of a
    level), within 1 level near one.  Bounds: an fp32 sum of 4096 squares in chunks of
    16 and a tree, relative error < 1e-5; flags exact where the oracle's bound is
    further than that from the limit."""
    import torch
    rng = np.random.default_rng(41)
    n, res, r = 16, 64, 320.0
    y = (rng.standard_normal((n, res, res, 5)) * 0.05).astype(np.float32)
    target = np.linspace(0.5, 3.5, n)                      # bounds around the 2 m limit
    y[..., 4] = (rng.standard_normal((n, res, res)) * (target * np.sqrt(2.0) / r)[:, None, None]).astype(np.float32)
    y[0, 3, 7, 4] = np.nan                                 # NaN bound -> fallback
    y[1, ..., 4] = -np.abs(y[1, ..., 4])                   # bound 0
    base = rng.random((n, res, res, 4)).astype(np.float32)
    base[..., 0] = (rng.standard_normal((n, res, res)) * 0.2).astype(np.float32)
    cz = (rng.standard_normal(n) * 300.0).astype(np.float32)
    fill_h = (rng.standard_normal((n, res, res)) * 50.0).astype(np.float32)
    fill_rgb = rng.integers(0, 256, (n, res, res, 3), dtype=np.uint8)
    region = synth.Region(tiles_x=4, tiles_y=4)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    inputs = {"base": T(base), "cz": T(cz), "fill_height": T(fill_h), "fill_rgb": T(fill_rgb)}
    h, c, bnd, fb = (t.cpu().numpy() for t in lsb.learned_finish(T(y), inputs, region, max_err_m=2.0))
    assert lsb.last_error() == 0
    hr, cr, br, fr = U.finish(y.astype(np.float64), base[..., 0].astype(np.float64), base[..., 1:].astype(np.float64),
                              cz.astype(np.float64), r, fill_h.astype(np.float64), fill_rgb, 2.0)
    assert np.isnan(bnd[0]) and np.isnan(br[0]) and fb[0] == 1 and fr[0] == 1
    assert bnd[1] == 0.0 and br[1] == 0.0
    np.testing.assert_allclose(bnd[1:], br[1:], rtol=1e-5, atol=0)
    decided = np.abs(br - 2.0) > 2e-5
    assert (fb[decided] == fr[decided]).all()
    assert 3 <= int(fr.sum()) <= n - 3                     # both branches exercised
    for o in range(n):
        if fr[o]:
            assert fb[o] == 1 and np.array_equal(h[o], fill_h[o]) and np.array_equal(c[o], fill_rgb[o])
            continue
        s = np.abs(base[o, ..., 0].astype(np.float64) + y[o, ..., 0])
        np.testing.assert_array_less(np.abs(h[o] - hr[o]), 2.0 ** -22 * (s * r + abs(float(cz[o]))) + 1e-7)
        v = np.clip(base[o, ..., 1:].astype(np.float64) + y[o, ..., 1:4], 0.0, 1.0) * 255.0 + 0.5
        safe = np.abs(v - np.round(v)) > 1e-4
        assert (c[o][safe] == cr[o][safe]).all()
        assert (np.abs(c[o].astype(int) - cr[o].astype(int)) <= 1).all()


def test_fill_learned_matches_oracle_chain(lsb):
    """The whole learned fill of 12 tiles (input raster, network, finish) against the
    oracle chain on the same bf16 weights: FP64 Gaussian fill, input raster, FP64
    network with bf16 storage, finish.  The error limit is set at the oracle's median
    bound, so both branches run.  Network tiles: relative L2 of the height residual
    (h - c_z)/r - base against the oracle's below 2e-2 (11 layers of bf16 storage,
    2^-9 each, as in the forward test) plus the fill's 1e-3 m; fallback tiles: the
    Gaussian fill within the fill bars; flags exact away from the limit (5 %, more
    than twice the forward bar)."""
    import torch
    from tests.helpers import assert_fill_close
    widths, n = (32, 64, 128), 12
    layers = U.layer_table(widths)
    rng = np.random.default_rng(43)
    params = U.init_params(43, layers)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.standard_normal(params[k].shape) * 0.05
    params["head.w"] *= 0.05                      # outputs of a few hundredths: errors in r, c_z show
    params["head.w"][4] *= 6.0                    # tile bounds spread over 12-25 m
    params["head.b"][4] = -0.02
    f = lsb.Filler(widths=widths, res=64, max_batch=8)
    f.params.copy_(torch.from_numpy(_flat(params, layers)))
    f.load()
    q = {}
    for name, ci, co, k in layers:
        w = params[name + ".w"].astype(np.float32)
        q[name + ".w"] = bf16_to_f64(bf16_bits(w)) if k == 3 else w.astype(np.float64)
        q[name + ".b"] = params[name + ".b"].astype(np.float32).astype(np.float64)
    region = synth.Region(tiles_x=5, tiles_y=4)
    counts = synth.lognormal_counts(44, 20)
    s = synth.region_samples(45, region, counts)
    tiles = np.array([0, 3, 6, 7, 8, 11, 12, 13, 14, 16, 18, 19], np.int64)
    ref = oracle.fill_sparse(s, region, tile_ids=tiles)
    xs, bh, bc, czs = [], [], [], []
    for o, t in enumerate(tiles):
        tx, ty = t % region.tiles_x, t // region.tiles_x
        a, b = s["tile_offsets"][t], s["tile_offsets"][t + 1]
        x, base_c, cz, r = U.tile_inputs(64, 64000, 1000, region.x0_cm + tx * 64000, region.y0_cm + ty * 64000,
                                         0.01, 0.0, 12000, s["x"][a:b], s["y"][a:b], s["z"][a:b], s["r"][a:b],
                                         s["g"][a:b], s["b"][a:b], ref["height"][o], ref["rgbf"][o],
                                         ref["nearest_d2"][o])
        xs.append(x); bh.append(x[..., 4]); bc.append(base_c); czs.append(cz)
    rnd = lambda a: bf16_to_f64(bf16_bits(a.astype(np.float32)))  # noqa: E731
    yr, _ = U.forward(q, rnd(np.stack(xs)), layers, store=rnd)
    bound0 = U.finish(yr, np.stack(bh), np.stack(bc), np.array(czs), r, ref["height"], ref["rgb8"], np.inf)[2]
    lim = float(np.median(bound0))
    hr, cr, br, fr = U.finish(yr, np.stack(bh), np.stack(bc), np.array(czs), r, ref["height"], ref["rgb8"], lim)
    h, c, bnd, fb = (t.cpu().numpy() for t in lsb.fill_learned(f, to_device(s), region, torch.as_tensor(tiles),
                                                               max_err_m=lim))
    assert lsb.last_error() == 0
    np.testing.assert_allclose(bnd, br, rtol=2e-2)
    decided = np.abs(br - lim) > 0.05 * lim
    assert decided.sum() >= 6 and (fb[decided] == fr[decided]).all()
    for o in np.nonzero(decided)[0]:
        if fr[o]:
            sub = {k: ref[k][o:o + 1] for k in ("height", "rgbf", "rgb8")}
            assert_fill_close(h[o:o + 1], c[o:o + 1], sub, msg=f"fallback tile {tiles[o]}")
            continue
        res_ref = (hr[o] - czs[o]) / r - bh[o]
        res_gpu = (h[o] - czs[o]) / r - bh[o]
        err = np.linalg.norm(res_gpu - res_ref) / np.linalg.norm(res_ref)
        assert err < 2e-2 + 1e-3 / (r * np.sqrt(np.mean(res_ref ** 2))), (tiles[o], err)
        assert np.abs(c[o].astype(int) - cr[o].astype(int)).mean() < 1.0, tiles[o]
