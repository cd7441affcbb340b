"""Training and evaluation of the learned filler on pairs the method generates itself.

Sec. 3.4 trains on ground-truth heightmaps made by taking the mean of all points that
fall onto a texel, with chunk points simulated as a sparse subsample; the pairs here
are (input raster of the chunk samples of a tile and its 8 neighbours, per-texel mean
of the tile's full-resolution points), both computed by this library's kernels.  The
optimiser is AdamW with a step schedule (Sec. 3.4); every forward and backward pass
runs in the library's tensor-core kernels through ``FillerFn``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import (Filler, FillerFn, PaperCNN, PaperCNNFn, adamw_step, bin_points, cnn_inputs, fill_interp, filler_loss,
               learned_inputs, learned_targets, learned_finish)


class FillerLossFn(torch.autograd.Function):
    """Loss of Sec. 3.4 (masked, clipped MSE + bound term) as [total, height, colour,
    bound]; backward (of the total) returns the kernel-computed dL/dy."""

    @staticmethod
    def forward(ctx, y, base, target, mask, bound_weight, bound_excess=False):
        loss, dy = filler_loss(y, base, target, mask, bound_weight, bound_excess)
        ctx.save_for_backward(dy)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dy,) = ctx.saved_tensors
        return dy * g[0], None, None, None, None, None


@dataclasses.dataclass
class TileSet:
    x: torch.Tensor        # bf16 bits int16 [n, res, res, 8]
    base: torch.Tensor     # [n, res, res, 4]
    target: torch.Tensor   # [n, res, res, 4]
    mask: torch.Tensor     # uint8 [n, res, res]
    cz: torch.Tensor       # [n]
    fill_height: torch.Tensor
    fill_rgb: torch.Tensor

    def __len__(self):
        return self.x.shape[0]


def synthetic_tiles(n_tiles, seed0, block=16, density=(3.0, 6.0), device="cuda"):
    """Pairs on seeded synthetic terrain: regions of (block+2)^2 tiles, one terrain seed
    each; inputs use the samples of all tiles, targets the full points of the inner
    block x block tiles only."""
    import synth
    import synth.gpu as sg
    parts = []
    made, r = 0, 0
    while made < n_tiles:
        seed = seed0 + r
        r += 1
        side = block + 2
        region = synth.Region(tiles_x=side, tiles_y=side)
        rng = np.random.default_rng(seed)
        dens = rng.uniform(density[0], density[1], side * side)
        counts = np.rint(dens * 640 * 640).astype(np.int64)
        inner = np.array([(ty * side + tx) for ty in range(1, side - 1) for tx in range(1, side - 1)], np.int64)
        samples = sg.region_samples(seed, region, counts, device=device)
        ids = torch.as_tensor(inner, dtype=torch.int32, device=device)
        inp = learned_inputs(samples, region, ids)
        full = np.zeros_like(counts)
        full[inner] = counts[inner]
        pts = sg.region_points(seed, region, full, device=device)
        (b64,), _ = bin_points(pts, region, levels=(64,))
        target, mask = learned_targets(b64, region, ids, inp["cz"])
        del pts, b64
        take = min(len(inner), n_tiles - made)
        parts.append(TileSet(inp["x"][:take], inp["base"][:take], target[:take], mask[:take], inp["cz"][:take],
                             inp["fill_height"][:take], inp["fill_rgb"][:take]))
        made += take
    cat = lambda k: torch.cat([getattr(p, k) for p in parts])  # noqa: E731
    return TileSet(*[cat(f.name) for f in dataclasses.fields(TileSet)])


LR = 1e-3  # learning rate of the short synthetic schedules (the paper: 1e-4 over 75 epochs)


def train(filler: Filler, data: TileSet, epochs=20, batch=256, lr=LR, weight_decay=1e-2, betas=(0.9, 0.999),
          eps=1e-5, milestones=(0.6, 0.85), gamma=0.1, bound_weight=1.0, seed=0, log=None, graph=None):
    """AdamW training with a step schedule; returns the per-epoch mean losses
    [total, height, colour, bound].  The bound channel learns the excess of the learned
    height's error over the Gaussian fill's (the finish step falls back to the Gaussian
    fill where that predicted excess is large).

    graph (default: on CUDA with more than one step): after one eager step, the batch
    gather, forward, loss and backward of a step run as one captured CUDA graph on
    static buffers (about 200 launches a step otherwise leave the eager loop bound by the
    host); AdamW, whose step count and rate change every step, stays outside.  The
    kernels and their order are those of the eager step, so the results are identical."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    p = filler.params
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    steps_per_epoch = max(1, len(data) // batch)
    total = epochs * steps_per_epoch
    if graph is None:
        graph = p.is_cuda and total > 1
    step = 0
    history = []
    idx_s = torch.empty(min(batch, len(data)), dtype=torch.int64, device=p.device)  # the graph's batch indices
    cap = None

    def forward_backward(idx):
        x = data.x[idx].contiguous()
        params = p.detach().requires_grad_(True)
        y = FillerFn.apply(params, x, filler)
        loss = FillerLossFn.apply(y, data.base[idx].contiguous(), data.target[idx].contiguous(),
                                  data.mask[idx].contiguous(), bound_weight, True)
        loss[0].backward()
        return loss.detach(), params.grad

    for ep in range(epochs):
        order = torch.randperm(len(data), generator=g).to(p.device)
        acc = torch.zeros(4, device=p.device)
        for k in range(steps_per_epoch):
            idx = order[k * batch:(k + 1) * batch]
            if graph and step > 0:
                if cap is None:
                    # capture once (the eager first step made every workspace and setting)
                    cap = torch.cuda.CUDAGraph()
                    side = torch.cuda.Stream()
                    side.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.stream(side):
                        with torch.cuda.graph(cap):
                            loss_s, grad_s = forward_backward(idx_s)
                    torch.cuda.current_stream().wait_stream(side)
                idx_s.copy_(idx)
                cap.replay()
                loss, grad = loss_s, grad_s
            else:
                loss, grad = forward_backward(idx)
            step += 1
            frac = step / total
            cur = lr * (gamma ** sum(frac > mm for mm in milestones))
            adamw_step(p, grad, m, v, step, lr=cur, betas=betas, eps=eps, weight_decay=weight_decay)
            acc += loss
        history.append([float(v) / steps_per_epoch for v in acc.tolist()])
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {history[-1]}")
    filler.load()
    return history


@torch.no_grad()
def evaluate(filler: Filler, data: TileSet, region_tile_cm=64000, z_scale=0.01, batch=None, max_err_m=2.0):
    """Height RMSE (m) and colour RMSE (8-bit levels) against the full-resolution means
    for the learned fill (the network alone, and with the Gaussian fallback above
    max_err_m) and the plain Gaussian fill, on texels with ground truth."""
    import types
    batch = batch or filler.max_batch
    r = 0.5 * region_tile_cm * z_scale
    reg = types.SimpleNamespace(x0_cm=0, y0_cm=0, tile_cm=region_tile_cm, tiles_x=1, tiles_y=1,
                                z_scale=z_scale, z_offset=0.0)
    se_l = se_f = se_g = se_lc = se_gc = 0.0
    cnt = 0.0
    fallbacks = 0
    for a in range(0, len(data), batch):
        sl = slice(a, a + batch)
        y = filler.forward(data.x[sl].contiguous())
        inp = {"base": data.base[sl].contiguous(), "cz": data.cz[sl].contiguous(),
               "fill_height": data.fill_height[sl].contiguous(), "fill_rgb": data.fill_rgb[sl].contiguous()}
        h, c, bound, fb = learned_finish(y, inp, reg, max_err_m=math.inf)
        hf, _, _, fbf = learned_finish(y, inp, reg, max_err_m=max_err_m)
        msk = data.mask[sl].bool()
        th = data.target[sl][..., 0] * r + data.cz[sl][:, None, None]
        tc = data.target[sl][..., 1:] * 255.0
        se_l += float(((h - th)[msk] ** 2).sum())
        se_f += float(((hf - th)[msk] ** 2).sum())
        se_g += float(((data.fill_height[sl] - th)[msk] ** 2).sum())
        se_lc += float(((c.float() - tc)[msk] ** 2).sum())
        se_gc += float(((data.fill_rgb[sl].float() - tc)[msk] ** 2).sum())
        cnt += float(msk.sum())
        fallbacks += int(fbf.sum())
    return {"height_rmse_learned_m": math.sqrt(se_l / cnt), "height_rmse_gaussian_m": math.sqrt(se_g / cnt),
            "height_rmse_with_fallback_m": math.sqrt(se_f / cnt), "max_err_m": max_err_m,
            "rgb_rmse_learned": math.sqrt(se_lc / (3 * cnt)), "rgb_rmse_gaussian": math.sqrt(se_gc / (3 * cnt)),
            "tiles": len(data), "fallback_tiles": fallbacks}


def init_params(filler: Filler, seed=0):
    """He-normal weights, zero biases; the head starts at zero (identity residual)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    flat = torch.zeros(filler.n_params)
    for cin, cout, k, w_off, b_off in filler.layers():
        n = cout * k * k * cin
        if k == 1:
            continue
        flat[w_off:w_off + n] = torch.randn(n, generator=g) * math.sqrt(2.0 / (cin * k * k))
    filler.params.copy_(flat.to(filler.params.device))
    filler.load()


# ------------------------------------------------------------------------------------
# the paper's network variant: Alg. 1 maps of the padded patch in, 64 x 64 out
# ------------------------------------------------------------------------------------

@dataclasses.dataclass
class PatchSet:
    x: torch.Tensor        # bf16 bits int16 [n, res, res, 8]
    target: torch.Tensor   # [n, 64, 64, 4]
    mask: torch.Tensor     # uint8 [n, 64, 64]
    cz: torch.Tensor       # [n]

    def __len__(self):
        return self.x.shape[0]


def patch_inputs(samples, region, tile_ids, res=128, stream=None):
    """Alg. 1 maps of the res x res patches (10 m texels: the tile plus (res - 64) / 2
    texels on every side) and the network input made from them."""
    pad = (res - 64) // 2 * (region.tile_cm // 64)
    maps = fill_interp(samples, region, tile_ids=tile_ids, res=res, pad_cm=pad,
                       maps=("nn_height", "nn_rgb", "lin_height", "lin_rgb"), stream=stream)
    x, cz = cnn_inputs(maps, r_m=0.5 * region.tile_cm * region.z_scale, stream=stream)
    return x, cz


def synthetic_patches(n_tiles, seed0, res=128, block=16, density=(3.0, 6.0), device="cuda"):
    """Training pairs of the paper's variant on seeded synthetic terrain (regions of
    (block + 4)^2 tiles, the inner block x block used: their padded patches see real
    samples all around)."""
    import synth
    import synth.gpu as sg
    parts, made, r = [], 0, 0
    while made < n_tiles:
        seed = seed0 + r
        r += 1
        side = block + 4
        region = synth.Region(tiles_x=side, tiles_y=side)
        rng = np.random.default_rng(seed)
        counts = np.rint(rng.uniform(density[0], density[1], side * side) * 640 * 640).astype(np.int64)
        inner = np.array([(ty * side + tx) for ty in range(2, side - 2) for tx in range(2, side - 2)], np.int64)
        samples = sg.region_samples(seed, region, counts, device=device)
        ids = torch.as_tensor(inner, dtype=torch.int32, device=device)
        x, cz = patch_inputs(samples, region, ids, res=res)
        full = np.zeros_like(counts)
        full[inner] = counts[inner]
        pts = sg.region_points(seed, region, full, device=device)
        (b64,), _ = bin_points(pts, region, levels=(64,))
        target, mask = learned_targets(b64, region, ids, cz)
        del pts, b64
        take = min(len(inner), n_tiles - made)
        parts.append(PatchSet(x[:take], target[:take], mask[:take], cz[:take]))
        made += take
    cat = lambda k: torch.cat([getattr(p, k) for p in parts])  # noqa: E731
    return PatchSet(*[cat(f.name) for f in dataclasses.fields(PatchSet)])


def train_cnn(cnn: PaperCNN, data: PatchSet, epochs=20, batch=256, lr=1e-3, weight_decay=1e-2, betas=(0.9, 0.999),
              eps=1e-5, milestones=(0.6, 0.85), gamma=0.1, bound_weight=1.0, seed=0, log=None, graph=None):
    """AdamW with a step schedule (Sec. 3.4) on the library's kernels; the outputs are
    the patch-space height and colours directly (zero base).  Returns per-epoch mean
    losses [total, height, colour, bound].  graph: the step after the first runs as a
    captured CUDA graph, as in train()."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    p = cnn.params
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    base = torch.zeros((batch,) + tuple(data.target.shape[1:]), dtype=torch.float32, device=p.device)
    steps_per_epoch = max(1, len(data) // batch)
    total = epochs * steps_per_epoch
    if graph is None:
        graph = p.is_cuda and total > 1
    step, history = 0, []
    idx_s = torch.empty(min(batch, len(data)), dtype=torch.int64, device=p.device)
    cap = None

    def forward_backward(idx):
        params = p.detach().requires_grad_(True)
        y = PaperCNNFn.apply(params, data.x[idx].contiguous(), cnn)
        loss = FillerLossFn.apply(y, base, data.target[idx].contiguous(), data.mask[idx].contiguous(),
                                  bound_weight)
        loss[0].backward()
        return loss.detach(), params.grad

    for ep in range(epochs):
        order = torch.randperm(len(data), generator=g).to(p.device)
        acc = torch.zeros(4, device=p.device)
        for k in range(steps_per_epoch):
            idx = order[k * batch:(k + 1) * batch]
            if graph and step > 0:
                if cap is None:
                    cap = torch.cuda.CUDAGraph()
                    side = torch.cuda.Stream()
                    side.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.stream(side):
                        with torch.cuda.graph(cap):
                            loss_s, grad_s = forward_backward(idx_s)
                    torch.cuda.current_stream().wait_stream(side)
                idx_s.copy_(idx)
                cap.replay()
                loss, grad = loss_s, grad_s
            else:
                loss, grad = forward_backward(idx)
            step += 1
            cur = lr * (gamma ** sum(step / total > mm for mm in milestones))
            adamw_step(p, grad, m, v, step, lr=cur, betas=betas, eps=eps, weight_decay=weight_decay)
            acc += loss
        history.append([float(v) / steps_per_epoch for v in acc.tolist()])
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {history[-1]}")
    cnn.load()
    return history


def init_cnn_params(cnn: PaperCNN, seed=0):
    """He-normal weights, zero biases; the head starts at zero.  The fully connected
    merge layers start at half the He scale: at full scale the four encoders' merged
    features kept the height loss on a plateau through the short schedule (held-out
    height loss 1.5e-3 after 30 epochs at lr 1e-3, against 7.4e-5 at half scale)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    flat = torch.zeros(cnn.n_params)
    for kind, cin, cout, w_off, b_off in cnn.layers():
        if kind == 2:
            continue
        fan = cin * (9 if kind == 0 else 1)
        scale = math.sqrt(2.0 / fan) * (0.5 if kind == 1 else 1.0)
        flat[w_off:w_off + cout * fan] = torch.randn(cout * fan, generator=g) * scale
    cnn.params.copy_(flat.to(cnn.params.device))
    cnn.load()
