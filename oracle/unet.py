"""FP64 numpy oracle of the learned filler: input raster, U-Net forward and backward,
loss and AdamW.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU baseline.  It shares no code with the CUDA path.

The paper refines interpolated heightmaps with a small U-Net-inspired CNN (Sec. 3.4),
normalises heights to patch space as (z - c_z) / r (Sec. 3.3 and 3.4), trains with an
MSE loss whose NaN-GT elements are zeroed and whose height and texture terms are
clipped to 0..1 and averaged, with AdamW (lr 1e-4, betas 0.9/0.999, eps 1e-5,
weight decay 1e-2) (Sec. 3.4).  The layer stack below is the 3-level 32/64/128
U-Net of the workload description; readings where the paper is silent:

* conv 3x3, stride 1, zero padding 1; ReLU after every 3x3 conv;
* 2x2 max pooling (ties: first in row-major window order gets the gradient);
* 2x nearest upsampling, skip concatenation as [upsampled, skip] along channels;
* a 1x1 head with 5 outputs: height residual, R, G, B residuals (added to the
  Gaussian-fill height and colour), and a predicted absolute height error;
* ReLU derivative at 0 is 0.
Layout: activations NHWC, weights [C_out][3][3][C_in] (OHWI), biases [C_out].
"""
from __future__ import annotations

import numpy as np

N_IN = 5
N_OUT = 5
BOUND_WEIGHT = 1.0


def layer_table(widths=(32, 64, 128), n_in=N_IN, n_out=N_OUT):
    """Layer list of an L-level U-Net with the given widths, L = len(widths).

    Encoder level l: conv 'e{l}a', conv 'e{l}b' (2x2 max pool between levels);
    decoder level l < L: upsample, concat with the encoder output of level l,
    conv 'd{l}a', conv 'd{l}b'; then the 1x1 'head'.  The default is the
    32/64/128 network; small widths give the tiny instances used for FD checks."""
    t = []
    cin = n_in
    for l, c in enumerate(widths, 1):
        t += [(f"e{l}a", cin, c, 3), (f"e{l}b", c, c, 3)]
        cin = c
    up = widths[-1]
    for l in range(len(widths) - 1, 0, -1):
        c = widths[l - 1]
        t += [(f"d{l}a", up + c, c, 3), (f"d{l}b", c, c, 3)]
        up = c
    t.append(("head", widths[0], n_out, 1))
    return tuple(t)


LAYERS = layer_table()


def param_count(layers=LAYERS):
    return sum(co * k * k * ci + co for _, ci, co, k in layers)


def init_params(seed, layers=LAYERS):
    """He-normal weights, zero biases (drawn with numpy's PCG64 from `seed`)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co, k in layers:
        std = np.sqrt(2.0 / (ci * k * k))
        p[name + ".w"] = rng.standard_normal((co, k, k, ci)) * std
        p[name + ".b"] = np.zeros(co)
    return p


# ------------------------------------------------------------------------------
# primitive ops (definitions written out; numpy tensordot is the only library step)
# ------------------------------------------------------------------------------

def conv(x, w, b):
    """out[n,y,x,o] = b[o] + sum_{ky,kx,i} xpad[n,y+ky,x+kx,i] w[o,ky,kx,i]."""
    k = w.shape[1]
    p = k // 2
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    out = np.zeros((n, h, wd, w.shape[0])) + b
    for ky in range(k):
        for kx in range(k):
            out += np.tensordot(xp[:, ky:ky + h, kx:kx + wd, :], w[:, ky, kx, :], axes=([3], [1]))
    return out


def conv_backward(x, w, dy):
    """Gradients of conv w.r.t. input, weight and bias."""
    k = w.shape[1]
    p = k // 2
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(k):
        for kx in range(k):
            dxp[:, ky:ky + h, kx:kx + wd, :] += np.tensordot(dy, w[:, ky, kx, :], axes=([3], [0]))
            dw[:, ky, kx, :] = np.tensordot(dy, xp[:, ky:ky + h, kx:kx + wd, :],
                                            axes=([0, 1, 2], [0, 1, 2]))
    dx = dxp[:, p:p + h, p:p + wd, :]
    return dx, dw, dy.sum(axis=(0, 1, 2))


def relu(x):
    return np.where(x > 0, x, 0.0)


def maxpool2(x):
    n, h, w, c = x.shape
    v = x.reshape(n, h // 2, 2, w // 2, 2, c)
    return v.max(axis=(2, 4))


def maxpool2_backward(x, dy):
    """Route each pooled gradient to the first maximum in row-major window order."""
    n, h, w, c = x.shape
    win = x.reshape(n, h // 2, 2, w // 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(n, h // 2, w // 2, 4, c)
    arg = win.argmax(axis=3)                        # first maximum
    dwin = np.zeros_like(win)
    np.put_along_axis(dwin, arg[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return dwin.reshape(n, h // 2, w // 2, 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(n, h, w, c)


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_backward(dy):
    n, h, w, c = dy.shape
    return dy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


# ------------------------------------------------------------------------------
# network
# ------------------------------------------------------------------------------

def _levels(layers):
    return sum(1 for name, *_ in layers if name.endswith("a") and name.startswith("e"))


def _identity(a):
    return a


def forward(params, x, layers=LAYERS, store=None):
    """Forward pass; returns (y, cache).  x: [N,H,W,C_in], H and W divisible by
    2^(L-1).  store: optional storage rounding applied to every conv output after
    its ReLU (arithmetic stays FP64; None keeps full precision)."""
    st = store or _identity
    L = _levels(layers)
    c = {"x": x}
    W = {name: (params[name + ".w"], params[name + ".b"]) for name, *_ in layers}
    h = x
    for l in range(1, L + 1):
        if l > 1:
            c[f"p{l - 1}"] = h = maxpool2(h)
        c[f"e{l}a"] = h = st(relu(conv(h, *W[f"e{l}a"])))
        c[f"e{l}b"] = h = st(relu(conv(h, *W[f"e{l}b"])))
    for l in range(L - 1, 0, -1):
        c[f"c{l}"] = h = np.concatenate([upsample2(h), c[f"e{l}b"]], axis=3)
        c[f"d{l}a"] = h = st(relu(conv(h, *W[f"d{l}a"])))
        c[f"d{l}b"] = h = st(relu(conv(h, *W[f"d{l}b"])))
    c["top"] = h
    y = conv(h, *W["head"])
    return y, c


def backward(params, cache, dy, layers=LAYERS, store=None):
    """Gradients of all parameters given dL/dy (hand-written chain rule).  store:
    optional storage rounding of every activation gradient passed between layers."""
    st = store or _identity
    L = _levels(layers)
    g = {}
    c = cache

    def conv_relu_back(name, xin, dout_post):
        # dout_post is dL/d(relu output); mask by the relu output
        dz = dout_post * (c[name] > 0)
        dx, g[name + ".w"], g[name + ".b"] = conv_backward(xin, params[name + ".w"], dz)
        return st(dx)

    d, g["head.w"], g["head.b"] = conv_backward(c["top"], params["head.w"], dy)
    d = st(d)
    skip = {}
    for l in range(1, L):
        d = conv_relu_back(f"d{l}b", c[f"d{l}a"], d)
        d = conv_relu_back(f"d{l}a", c[f"c{l}"], d)
        cu = d.shape[3] - c[f"e{l}b"].shape[3]
        skip[l] = d[..., cu:]
        d = st(upsample2_backward(d[..., :cu]))
    for l in range(L, 0, -1):
        if l < L:
            d = st((maxpool2_backward(c[f"e{l}b"], d) + skip[l]) * (c[f"e{l}b"] > 0))
        d = conv_relu_back(f"e{l}b", c[f"e{l}a"], d)
        d = conv_relu_back(f"e{l}a", c[f"p{l - 1}"] if l > 1 else c["x"], d)
    return g


# ------------------------------------------------------------------------------
# loss (Sec. 3.4): masked, clipped MSE on height and colour, averaged; plus the
# squared-error regression of the error-bound channel onto a (detached) error target
# (a reading: the paper has no bound), on the height term's scale.  The target is the
# absolute height error |e|, or, with bound_excess, the excess max(|e| - |e_base|, 0)
# of the learned height's error over the base fill's error e_base = base_h - t_h.
# ------------------------------------------------------------------------------

def loss_and_grad(y, base_h, base_c, t_h, t_c, mask, bound_weight=BOUND_WEIGHT, bound_excess=False):
    """y: [N,H,W,5] net output; base_h [N,H,W], base_c [N,H,W,3] the Gaussian-fill
    inputs the residuals are added to; t_h, t_c targets; mask [N,H,W] in {0,1}.
    Returns (loss, dL/dy, parts)."""
    m = mask.astype(np.float64)
    cnt = max(m.sum(), 1.0)
    eh = base_h + y[..., 0] - t_h
    ec = base_c + y[..., 1:4] - t_c
    sh, sc = eh * eh, ec * ec
    lh = (np.minimum(sh, 1.0) * m).sum() / cnt
    lc = (np.minimum(sc, 1.0) * m[..., None]).sum() / (3.0 * cnt)
    tb = np.abs(eh)                                  # detached target
    if bound_excess:
        tb = np.maximum(tb - np.abs(base_h - t_h), 0.0)
    db = y[..., 4] - tb
    lb = (db * db * m).sum() / cnt
    loss = 0.5 * (lh + lc) + bound_weight * lb
    dy = np.zeros_like(y)
    dy[..., 0] = 0.5 * 2.0 * eh * (sh < 1.0) * m / cnt
    dy[..., 1:4] = 0.5 * 2.0 * ec * (sc < 1.0) * m[..., None] / (3.0 * cnt)
    dy[..., 4] = bound_weight * 2.0 * db * m / cnt
    return loss, dy, {"height": lh, "color": lc, "bound": lb}


def adamw_step(p, g, m, v, step, lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-5, wd=1e-2):
    """One AdamW update (decoupled weight decay), in place; step counts from 1."""
    p *= (1.0 - lr * wd)
    m[...] = beta1 * m + (1.0 - beta1) * g
    v[...] = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------------------
# learned-filler input raster (5 channels) from the fill results of one tile
# ------------------------------------------------------------------------------

def tile_inputs(res, tile_cm, cell_cm, tile_x0, tile_y0, z_scale, z_offset, radius_cm,
                sx, sy, sz, sr, sg, sb, fill_h, fill_c, nearest_d2):
    """Input channels of one tile (patch-space normalisation of Sec. 3.3/3.4):

    r = tile_cm/2 in metres; c_z = mean Gaussian-fill height of the 4 central texels;
    ch0 = (z_s - c_z)/r at texels holding a sample of this tile (lowest sample
          index wins), else 0;
    ch1 = luma (0.299 R + 0.587 G + 0.114 B)/65535 of that sample, else 0;
    ch2 = 1 where a sample lies in the texel, else 0;
    ch3 = min(sqrt(nearest_d2), 2R) / R;
    ch4 = (fill height - c_z)/r.
    Returns (x [res,res,5], base_c [res,res,3] Gaussian colour in 0..1, c_z, r)."""
    r_m = 0.5 * tile_cm * z_scale
    c = res // 2
    cz = fill_h[c - 1:c + 1, c - 1:c + 1].mean()
    x = np.zeros((res, res, 5))
    for s in range(len(sx) - 1, -1, -1):                 # lowest index written last
        lx, ly = int(sx[s]) - tile_x0, int(sy[s]) - tile_y0
        if not (0 <= lx < tile_cm and 0 <= ly < tile_cm):
            continue
        i, j = ly // cell_cm, lx // cell_cm
        zm = float(sz[s]) * z_scale + z_offset
        x[i, j, 0] = (zm - cz) / r_m
        x[i, j, 1] = (0.299 * float(sr[s]) + 0.587 * float(sg[s]) + 0.114 * float(sb[s])) / 65535.0
        x[i, j, 2] = 1.0
    d = np.sqrt(nearest_d2.astype(np.float64))
    x[..., 3] = np.minimum(d, 2.0 * radius_cm) / radius_cm
    x[..., 4] = (fill_h - cz) / r_m
    base_c = fill_c * 256.0 / 65535.0
    return x, base_c, cz, r_m


# ------------------------------------------------------------------------------
# finish (step a11): de-normalisation of the network output, the per-tile error
# bound and the Gaussian fallback
# ------------------------------------------------------------------------------

def finish(y, base_h, base_c, cz, r_m, fill_h, fill_rgb, max_err_m):
    """Final heights and 8-bit colours of a batch of tiles from the network output.

    y [N,H,W,5] network output (residuals 0..3, error channel 4); base_h [N,H,W] the
    Gaussian-fill height in patch space (fill - c_z)/r; base_c [N,H,W,3] the
    Gaussian-fill colour in 0..1; cz [N] the patch centres in metres; r_m the patch
    half side in metres; fill_h [N,H,W], fill_rgb [N,H,W,3] the Gaussian fill itself.

    * de-normalisation (Sec. 3.3/3.4: patch space is (z - c_z)/r, so z = z'·r + c_z):
      height = (base_h + y0)·r + c_z;
    * colour: c = base_c + y1..3, clamped to 0..1, 8 bits by round half up of c·255;
    * error bound (a reading; the paper has none): the root mean square of the
      clamped error channel max(y4, 0) over the tile's texels, times r (a NaN in
      the channel makes the bound NaN);
    * fallback: a tile whose bound is not <= max_err_m (above it, or NaN) takes the
      Gaussian fill unchanged.
    Returns (height, rgb8, bound [N], used_fallback [N] in {0, 1})."""
    n = y.shape[0]
    height = np.empty(base_h.shape)
    rgb = np.empty(base_c.shape, dtype=np.uint8)
    bound = np.empty(n)
    used = np.empty(n, dtype=np.uint8)
    for o in range(n):
        e = np.where(y[o, ..., 4] < 0.0, 0.0, y[o, ..., 4])  # a NaN output stays NaN
        bound[o] = np.sqrt(np.mean(e * e)) * r_m
        used[o] = 0 if bound[o] <= max_err_m else 1
        if used[o]:
            height[o] = fill_h[o]
            rgb[o] = fill_rgb[o]
            continue
        height[o] = (base_h[o] + y[o, ..., 0]) * r_m + cz[o]
        c = np.clip(base_c[o] + y[o, ..., 1:4], 0.0, 1.0)
        rgb[o] = np.floor(c * 255.0 + 0.5).astype(np.uint8)
    return height, rgb, bound, used
