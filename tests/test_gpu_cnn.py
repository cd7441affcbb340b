"""GPU parity of the paper's network variant (tensor-core convolutions, fp32 fully
connected layers) against the FP64 oracle/cnn.py: the layer table, the forward output
(relative L2 < 3e-2: bf16 activations through 13 layers on the longest path), every
layer's parameter gradient (relative L2 < 2e-2 with every ReLU active; direction only
with random signs, where bf16 rounding flips the ReLU branch of near-zero units), the
input raster, bit-reproducible gradients, and AdamW steps that reduce the loss."""
import numpy as np
import pytest

import oracle.cnn as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    return lsb


def _bf16(a):
    import torch
    t = torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16)
    return t.float().numpy().astype(np.float64), t.view(torch.int16)


def _setup(lsb, res=32, n=32, seed=0):
    import torch
    cnn = lsb.PaperCNN(res=res, max_batch=n)
    p = C.init_params(seed, res)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    cnn.params.copy_(torch.as_tensor(C.flatten(p, res), dtype=torch.float32))
    xf, xb = _bf16(rng.standard_normal((n, res, res, 8)) * 0.5)
    return cnn, p, xf, xb.cuda()


@pytest.mark.parametrize("res", [32, 64, 128])
def test_layer_table_matches_oracle(lsb, res):
    cnn = lsb.PaperCNN(res=res, max_batch=32, training=False)
    table = C.layer_table(res)
    kinds = {"conv": 0, "fc": 1, "head": 2}
    off = 0
    got = cnn.layers()
    assert len(got) == len(table)
    for (name, kind, ci, co), (k, gci, gco, wo, bo) in zip(table, got):
        assert (k, gci, gco) == (kinds[kind], ci, co), name
        assert wo == off, name
        off += co * ci * (9 if kind == "conv" else 1)
        assert bo == off, name
        off += co
    assert cnn.n_params == C.param_count(res) == off


def test_forward_matches_oracle(lsb):
    import torch
    cnn, p, xf, xb = _setup(lsb)
    cnn.load()
    y = cnn.forward(xb).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    ref, _ = C.forward(p, xf)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel < 3e-2, rel


def _grads(lsb, cnn, p, xf, xb, seed=9):
    import torch
    cnn.load()
    y = cnn.forward(xb)
    gy = np.random.default_rng(seed).standard_normal(tuple(y.shape))
    g = cnn.backward(torch.as_tensor(gy, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    _, cache = C.forward(p, xf)
    return C.unflatten(g.cpu().numpy().astype(np.float64), cnn.res), C.backward(p, cache, gy), g


def _compare(got, ref, res, max_rel, min_cos, exclude=()):
    for name, *_ in C.layer_table(res):
        for part in (".w", ".b"):
            a, b = got[name + part].ravel(), ref[name + part].ravel()
            nb = np.linalg.norm(b)
            if nb == 0 or name in exclude:
                continue
            rel = np.linalg.norm(a - b) / nb
            cos = float(a @ b / (np.linalg.norm(a) * nb))
            assert rel < max_rel and cos > min_cos, (name + part, rel, cos)


@pytest.mark.parametrize("res,n", [(32, 32), (128, 2)])
def test_gradients_match_oracle_with_every_relu_active(lsb, res, n):
    """Non-negative inputs and weights and positive biases keep every pre-activation
    positive, so no ReLU mask depends on rounding: every layer's gradient then agrees
    with the FP64 oracle to bf16 precision (rel. L2 < 2e-2; the layers behind a max pool
    also see the rare routing changes of near-equal bf16 values).  At res 128 the
    full-resolution layers run the weight gradient in half-row stages."""
    import torch
    cnn = lsb.PaperCNN(res=res, max_batch=n)
    p = C.init_params(3, res)
    for k in p:
        p[k] = np.full(p[k].shape, 0.1) if k.endswith(".b") else np.abs(p[k]) * 0.5
    cnn.params.copy_(torch.as_tensor(C.flatten(p, res), dtype=torch.float32))
    xf, xb = _bf16(np.abs(np.random.default_rng(4).standard_normal((n, res, res, 8))) * 0.5)
    got, ref, _ = _grads(lsb, cnn, p, xf, xb.cuda())
    _compare(got, ref, res, 2e-2, 0.9999)


def test_gradients_general_weights_and_reproducible(lsb):
    """Random signs: units whose pre-activation lies within bf16 rounding of zero take a
    different ReLU branch than in FP64, and the L2 error grows with the square root of
    that fraction through the 17 layers from the loss to the first encoder layer; the
    direction stays (cosine > 0.95), the head and the final CNN agree closely, and two
    backward passes are bit-identical."""
    import torch
    cnn, p, xf, xb = _setup(lsb, seed=3)
    got, ref, g1 = _grads(lsb, cnn, p, xf, xb)
    _, _, g2 = _grads(lsb, cnn, p, xf, xb)
    assert torch.equal(g1, g2)
    _compare(got, ref, 32, 0.4, 0.95)
    _compare(got, ref, 32, 1e-1, 0.995, exclude=[n for n, *_ in C.layer_table(32) if not n.startswith(("head", "f."))])


def test_inputs_match_oracle(lsb):
    import torch
    rng = np.random.default_rng(4)
    n, res = 3, 32
    lin = rng.uniform(300, 700, (n, res, res)).astype(np.float32)
    nn = (lin + rng.normal(0, 2, lin.shape)).astype(np.float32)
    lin[1, 0, :4] = np.nan
    lr, nr = (rng.integers(0, 256, (n, res, res, 3)).astype(np.uint8) for _ in range(2))
    maps = {"lin_height": torch.as_tensor(lin).cuda(), "nn_height": torch.as_tensor(nn).cuda(),
            "lin_rgb": torch.as_tensor(lr).cuda(), "nn_rgb": torch.as_tensor(nr).cuda()}
    x, cz = lsb.cnn_inputs(maps, r_m=320.0)
    xr, czr = C.inputs(lin.astype(np.float64), nn.astype(np.float64), lr.astype(np.float64),
                       nr.astype(np.float64), 320.0)
    np.testing.assert_allclose(cz.cpu().numpy(), czr, rtol=1e-6)
    xg = x.view(torch.bfloat16).float().cpu().numpy()
    np.testing.assert_allclose(xg, xr, rtol=2 ** -8, atol=1e-6)


def test_adamw_steps_reduce_the_loss(lsb):
    import torch
    cnn, p, xf, xb = _setup(lsb, seed=5)
    n, c = 32, 16
    rng = np.random.default_rng(6)
    target = torch.as_tensor(rng.uniform(-0.2, 0.2, (n, c, c, 4)), dtype=torch.float32, device="cuda")
    base = torch.zeros_like(target)
    mask = torch.ones((n, c, c), dtype=torch.uint8, device="cuda")
    m = torch.zeros_like(cnn.params)
    v = torch.zeros_like(cnn.params)
    losses = []
    for step in range(1, 31):
        cnn.load()
        y = cnn.forward(xb)
        loss, dy = lsb.filler_loss(y, base, target, mask)
        g = cnn.backward(dy)
        lsb.adamw_step(cnn.params, g, m, v, step, lr=1e-3)
        losses.append(float(loss[0]))
    assert lsb.last_error() == 0
    assert losses[-1] < 0.5 * losses[0], losses


def test_graph_captured_cnn_training_is_bit_identical_to_eager(lsb):
    """train_cnn with the step captured as a CUDA graph (after one eager step) against
    the eager loop: identical parameters and losses after two epochs."""
    import torch
    from paper_2509_20198_b300 import train as T
    data = T.synthetic_patches(64, seed0=310, res=128, block=4)
    out = []
    for graph in (False, True):
        cnn = lsb.PaperCNN(res=128, max_batch=16)
        T.init_cnn_params(cnn, seed=7)
        hist = T.train_cnn(cnn, data, epochs=2, batch=16, lr=T.LR, graph=graph)
        torch.cuda.synchronize()
        assert lsb.last_error() == 0
        out.append((cnn.params.clone(), hist))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
