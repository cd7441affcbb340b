"""Pins of the paper-variant network oracle (oracle/cnn.py): central finite differences
for the whole backward pass, the independence of the four encoders, the skip path that
carries the raw inputs to the final CNN, the crop, and the input normalisation."""
import numpy as np
import pytest

import oracle.cnn as C
import oracle.unet as U


def test_parameter_count_is_the_papers_two_and_a_half_million():
    assert C.param_count(128) == 2_481_733
    v = C.flatten(C.init_params(0, 128), 128)
    assert v.size == C.param_count(128)
    p = C.unflatten(v, 128)
    assert p["fc2.w"].shape == (1024, 1024) and p["head.w"].shape == (5, 1, 1, 16)


def test_backward_matches_finite_differences():
    res, n, h = 32, 2, 1e-6
    rng = np.random.default_rng(0)
    p = C.init_params(0, res)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((n, res, res, 8))
    gy = rng.standard_normal((n, res // 2, res // 2, 5))

    def f(q):
        y, _ = C.forward(q, x)
        return float((y * gy).sum())

    _, cache = C.forward(p, x)
    g = C.backward(p, cache, gy)
    worst = 0.0
    for k in p:
        flat = p[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(flat.size, 6), replace=False):
            old = flat[i]
            flat[i] = old + h
            fp = f(p)
            flat[i] = old - h
            fm = f(p)
            flat[i] = old
            fd = (fp - fm) / (2 * h)
            an = g[k].reshape(-1)[i]
            worst = max(worst, abs(fd - an) / max(1.0, abs(fd), abs(an)))
    assert worst < 1e-6


def test_encoders_are_independent():
    """Changing the NN-height channel changes only encoder 1's features."""
    res = 32
    p = C.init_params(1, res)
    x = np.random.default_rng(2).standard_normal((2, res, res, 8))
    _, c0 = C.forward(p, x)
    x2 = x.copy()
    x2[..., 1] += 0.5
    _, c1 = C.forward(p, x2)
    for k in range(4):
        same = np.array_equal(c0[f"fc1.{k}.out"], c1[f"fc1.{k}.out"])
        assert same == (k != 1), k


def test_skip_path_carries_the_inputs():
    """With the fully connected layers zeroed the decoders see a constant, and the
    final CNN's output at a texel depends on the raw inputs through the concat: the
    result equals the final CNN applied to [x, Dh, Dt] computed by hand."""
    res = 32
    p = C.init_params(3, res)
    for k in list(p):
        if k.startswith("fc"):
            p[k] = np.zeros_like(p[k])
    x = np.random.default_rng(4).standard_normal((1, res, res, 8))
    y, _ = C.forward(p, x)
    dec = []
    for j in ("h", "t"):
        a = np.zeros((1, res // 16, res // 16, 16))
        for l in range(5):
            a = U.relu(U.conv(a, p[f"d{j}.{l}.w"], p[f"d{j}.{l}.b"]))
            a = U.upsample2(a) if l < 4 else a
        dec.append(a)
    a = np.concatenate([x] + dec, axis=-1)
    for l in range(2):
        a = U.relu(U.conv(a, p[f"f.{l}.w"], p[f"f.{l}.b"]))
    full = U.conv(a, p["head.w"], p["head.b"])
    np.testing.assert_allclose(y, full[:, 8:24, 8:24, :], rtol=1e-12, atol=1e-12)
    x2 = x.copy()
    x2[0, 16, 16, 3] += 1.0  # a colour input reaches the output only through the skip
    y2, _ = C.forward(p, x2)
    assert not np.allclose(y, y2)


def test_inputs_normalisation_hand_case():
    res = 4
    lin = np.arange(16, dtype=np.float64).reshape(1, 4, 4) + 100.0
    nn = lin + 1.0
    rgb = np.full((1, 4, 4, 3), 51.0)
    x, cz = C.inputs(lin, nn, rgb, rgb * 2, r_m=320.0)
    assert cz[0] == pytest.approx((105 + 106 + 109 + 110) / 4)
    assert x[0, 0, 0, 0] == pytest.approx((100 - cz[0]) / 320.0)
    assert x[0, 0, 0, 1] == pytest.approx((101 - cz[0]) / 320.0)
    assert x[0, 2, 3, 2] == pytest.approx(0.2) and x[0, 2, 3, 7] == pytest.approx(0.4)
    lin[0, 0, 0] = np.nan
    x, _ = C.inputs(lin, nn, rgb, rgb, r_m=320.0)
    assert x[0, 0, 0, 0] == 0.0
