"""FP64 numpy oracle of the paper's own network variant (Sec. 3.4): per-input encoders,
two fully connected merge steps, two decoders (height and texture), one skip
connection that concatenates the original inputs with the decoder outputs, a final
CNN, and the centre crop.

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing in the product path.  It
shares no code with the CUDA path (the convolution, pooling, upsampling, loss and
AdamW definitions come from oracle.unet).

The text names the parts but not their sizes (its architecture figure is not in the
text); the readings, sized to the paper's 2.5M parameters at res 128:

* input: res x res texels with 8 channels: linear height, NN height (patch space),
  linear RGB, NN RGB (0..1); the four inputs are encoded independently;
* encoder of one input: four times (3x3 conv + ReLU, 2x2 max pool) with 16, 32, 64,
  64 channels, then a 3x3 conv + ReLU to 16 channels at res / 16; flattened in NHWC
  order;
* merge step 1: per input a fully connected layer to 256 + ReLU; step 2: the four
  concatenated (1024) to 16 * (res / 16)^2 + ReLU, reshaped to [res/16, res/16, 16];
* decoder (height and texture separately): 3x3 conv + ReLU with 64, 32, 32, 16
  channels, each followed by 2x nearest upsampling, then a 3x3 conv + ReLU with 16;
* skip: concat [input (8), height decoder (16), texture decoder (16)] = 40 channels;
* final CNN: 3x3 conv + ReLU to 32 and to 16, then a 1x1 head to 5 outputs (height,
  R, G, B and the error bound of the learned filler); the output is the centre
  res/2 x res/2 crop (64 x 64 of 128).
Layout: weights of conv layers [C_out][k][k][C_in] (OHWI), of fully connected ones
[out][in]; each layer's bias follows its weights in the flat parameter vector.
"""
from __future__ import annotations

import numpy as np

from . import unet as U

IN_CH = 8
ENC_IN = ((0, 1), (1, 1), (2, 3), (5, 3))  # (first channel, channels) of each input
ENC_W = (16, 32, 64, 64)
ENC_OUT = 16
FC1 = 256
DEC_W = (64, 32, 32, 16, 16)
FIN_W = (32, 16)
N_OUT = 5
CAT = IN_CH + 2 * DEC_W[-1]


def layer_table(res=128):
    """[(name, kind, cin, cout)], kind 'conv' (3x3), 'fc' or 'head' (1x1)."""
    b = res // 16
    t = []
    for k, (_, ck) in enumerate(ENC_IN):
        cin = ck
        for l, c in enumerate(ENC_W):
            t.append((f"e{k}.{l}", "conv", cin, c))
            cin = c
        t.append((f"e{k}.4", "conv", cin, ENC_OUT))
    for k in range(4):
        t.append((f"fc1.{k}", "fc", ENC_OUT * b * b, FC1))
    t.append(("fc2", "fc", 4 * FC1, ENC_OUT * b * b))
    for j in ("h", "t"):
        cin = ENC_OUT
        for l, c in enumerate(DEC_W):
            t.append((f"d{j}.{l}", "conv", cin, c))
            cin = c
    t.append(("f.0", "conv", CAT, FIN_W[0]))
    t.append(("f.1", "conv", FIN_W[0], FIN_W[1]))
    t.append(("head", "head", FIN_W[1], N_OUT))
    return t


def _wshape(kind, cin, cout):
    return (cout, 3, 3, cin) if kind == "conv" else ((cout, 1, 1, cin) if kind == "head" else (cout, cin))


def param_count(res=128):
    return sum(int(np.prod(_wshape(k, ci, co))) + co for _, k, ci, co in layer_table(res))


def init_params(seed, res=128):
    """He-normal weights, zero biases (numpy PCG64 from `seed`)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, kind, ci, co in layer_table(res):
        fan = ci * (9 if kind == "conv" else 1)
        p[name + ".w"] = rng.standard_normal(_wshape(kind, ci, co)) * np.sqrt(2.0 / fan)
        p[name + ".b"] = np.zeros(co)
    return p


def flatten(p, res=128):
    return np.concatenate([np.concatenate([p[n + ".w"].ravel(), p[n + ".b"]]) for n, *_ in layer_table(res)])


def unflatten(v, res=128):
    p, o = {}, 0
    for name, kind, ci, co in layer_table(res):
        s = _wshape(kind, ci, co)
        k = int(np.prod(s))
        p[name + ".w"] = v[o:o + k].reshape(s)
        o += k
        p[name + ".b"] = v[o:o + co]
        o += co
    return p


def crop(res):
    """(offset, size) of the output crop."""
    return res // 4, res // 2


def forward(p, x):
    """x [N, res, res, 8] -> (y [N, res/2, res/2, 5], cache)."""
    n, res = x.shape[0], x.shape[1]
    b = res // 16
    cache = {"x": x}
    h1 = []
    for k, (c0, ck) in enumerate(ENC_IN):
        a = x[..., c0:c0 + ck]
        for l in range(4):
            z = U.relu(U.conv(a, p[f"e{k}.{l}.w"], p[f"e{k}.{l}.b"]))
            cache[f"e{k}.{l}.in"], cache[f"e{k}.{l}.out"] = a, z
            a = U.maxpool2(z)
        z = U.relu(U.conv(a, p[f"e{k}.4.w"], p[f"e{k}.4.b"]))
        cache[f"e{k}.4.in"], cache[f"e{k}.4.out"] = a, z
        f = z.reshape(n, -1)
        h = U.relu(f @ p[f"fc1.{k}.w"].T + p[f"fc1.{k}.b"])
        cache[f"fc1.{k}.in"], cache[f"fc1.{k}.out"] = f, h
        h1.append(h)
    zc = np.concatenate(h1, axis=1)
    g = U.relu(zc @ p["fc2.w"].T + p["fc2.b"])
    cache["fc2.in"], cache["fc2.out"] = zc, g
    dec = []
    for j in ("h", "t"):
        a = g.reshape(n, b, b, ENC_OUT)
        for l in range(5):
            z = U.relu(U.conv(a, p[f"d{j}.{l}.w"], p[f"d{j}.{l}.b"]))
            cache[f"d{j}.{l}.in"], cache[f"d{j}.{l}.out"] = a, z
            a = U.upsample2(z) if l < 4 else z
        dec.append(a)
    cat = np.concatenate([x, dec[0], dec[1]], axis=-1)
    a = cat
    for l in range(2):
        z = U.relu(U.conv(a, p[f"f.{l}.w"], p[f"f.{l}.b"]))
        cache[f"f.{l}.in"], cache[f"f.{l}.out"] = a, z
        a = z
    yfull = U.conv(a, p["head.w"], p["head.b"])
    cache["head.in"] = a
    o, c = crop(res)
    return yfull[:, o:o + c, o:o + c, :], cache


def backward(p, cache, dy):
    """Gradients (dict like p) of all parameters given dL/dy of the cropped output."""
    x = cache["x"]
    n, res = x.shape[0], x.shape[1]
    b = res // 16
    g = {}
    o, c = crop(res)
    dyf = np.zeros((n, res, res, N_OUT))
    dyf[:, o:o + c, o:o + c, :] = dy
    da, g["head.w"], g["head.b"] = U.conv_backward(cache["head.in"], p["head.w"], dyf)
    for l in (1, 0):
        dz = da * (cache[f"f.{l}.out"] > 0)
        da, g[f"f.{l}.w"], g[f"f.{l}.b"] = U.conv_backward(cache[f"f.{l}.in"], p[f"f.{l}.w"], dz)
    dcat = da
    dg = np.zeros((n, b, b, ENC_OUT))
    for jj, j in enumerate(("h", "t")):
        da = dcat[..., IN_CH + 16 * jj:IN_CH + 16 * (jj + 1)]
        for l in (4, 3, 2, 1, 0):
            if l < 4:
                da = U.upsample2_backward(da)
            dz = da * (cache[f"d{j}.{l}.out"] > 0)
            da, g[f"d{j}.{l}.w"], g[f"d{j}.{l}.b"] = U.conv_backward(cache[f"d{j}.{l}.in"], p[f"d{j}.{l}.w"], dz)
        dg += da
    dg2 = dg.reshape(n, -1) * (cache["fc2.out"] > 0)
    g["fc2.w"] = dg2.T @ cache["fc2.in"]
    g["fc2.b"] = dg2.sum(axis=0)
    dzc = dg2 @ p["fc2.w"]
    for k in range(4):
        dh = dzc[:, FC1 * k:FC1 * (k + 1)] * (cache[f"fc1.{k}.out"] > 0)
        g[f"fc1.{k}.w"] = dh.T @ cache[f"fc1.{k}.in"]
        g[f"fc1.{k}.b"] = dh.sum(axis=0)
        da = (dh @ p[f"fc1.{k}.w"]).reshape(n, b, b, ENC_OUT)
        for l in (4, 3, 2, 1, 0):
            if l < 4:
                da = U.maxpool2_backward(cache[f"e{k}.{l}.out"], da)
            dz = da * (cache[f"e{k}.{l}.out"] > 0)
            da, g[f"e{k}.{l}.w"], g[f"e{k}.{l}.b"] = U.conv_backward(cache[f"e{k}.{l}.in"], p[f"e{k}.{l}.w"], dz)
    return g


def inputs(lin_h, nn_h, lin_rgb8, nn_rgb8, r_m):
    """Network input [N, res, res, 8] and c_z [N] from the Alg. 1 maps of N patches
    (heights in metres, colours 8-bit): heights (z - c_z) / r with c_z the mean of the
    linear map's 4 central texels (the patch centre of an even grid), colours / 255.
    A texel without a height (an empty window) is 0."""
    n, res = lin_h.shape[0], lin_h.shape[1]
    m = res // 2
    cz = lin_h[:, m - 1:m + 1, m - 1:m + 1].reshape(n, 4).mean(axis=1)
    x = np.zeros((n, res, res, IN_CH))
    x[..., 0] = (lin_h - cz[:, None, None]) / r_m
    x[..., 1] = (nn_h - cz[:, None, None]) / r_m
    x[..., 2:5] = lin_rgb8 / 255.0
    x[..., 5:8] = nn_rgb8 / 255.0
    return np.nan_to_num(x, nan=0.0), cz
