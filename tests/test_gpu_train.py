"""Training of the learned filler on the GPU (tensor-core forward and backward through
FillerFn) on pairs the method generates itself, and what it gains over the plain
Gaussian fill on held-out terrain seeds (height RMSE against the full-resolution
per-texel means, Sec. 3.4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    return lsb


def test_fillerfn_gradient_equals_native_backward(lsb):
    import torch
    from paper_2509_20198_b300 import train as T
    f = lsb.Filler(max_batch=2)
    T.init_params(f, seed=3)
    f.params[-5:] = 0.01
    x = torch.zeros((2, 64, 64, 8), dtype=torch.int16, device="cuda")
    x[..., :5] = torch.randn((2, 64, 64, 5), device="cuda").to(torch.bfloat16).view(torch.int16)
    p = f.params.detach().requires_grad_(True)
    y = lsb.FillerFn.apply(p, x, f)
    w = torch.randn_like(y)
    (y * w).sum().backward()
    g2 = f.backward(w)
    # every reduction of the backward pass runs in a fixed order: bit-identical
    assert torch.equal(p.grad, g2)


def test_graph_captured_training_step_is_bit_identical_to_eager(lsb):
    """The captured step (gather, forward, loss, backward as one CUDA graph, AdamW
    outside) replays the eager step's kernels in the same order: after several steps
    and an epoch boundary the parameters and losses are bit-identical."""
    import torch
    from paper_2509_20198_b300 import train as T
    data = T.synthetic_tiles(96, seed0=300)
    out = []
    for graph in (False, True):
        f = lsb.Filler(max_batch=32)
        T.init_params(f, seed=5)
        hist = T.train(f, data, epochs=2, batch=32, lr=T.LR, graph=graph)
        torch.cuda.synchronize()
        assert lsb.last_error() == 0
        out.append((f.params.clone(), hist))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_training_beats_gaussian_fill_on_held_out_tiles(lsb):
    import torch
    from paper_2509_20198_b300 import train as T
    train_set = T.synthetic_tiles(4096, seed0=100)
    held = T.synthetic_tiles(256, seed0=900)
    f = lsb.Filler(max_batch=256)
    T.init_params(f, seed=0)
    before = T.evaluate(f, held)
    # every gradient reduction runs in a fixed order, so this training is reproducible
    # run to run (observed: learned / Gaussian height RMSE = 0.76)
    hist = T.train(f, train_set, epochs=60, batch=256, lr=T.LR)
    after = T.evaluate(f, held)
    torch.cuda.synchronize()
    assert lsb.last_error() == 0
    print("before", before, "after", after, "loss", hist[0], hist[-1])
    # the zero-initialised head starts as the Gaussian fill itself
    assert before["height_rmse_learned_m"] == pytest.approx(before["height_rmse_gaussian_m"], rel=1e-3)
    assert hist[-1][0] < hist[0][0] and hist[-1][1] < hist[0][1]
    assert after["height_rmse_learned_m"] < 0.9 * after["height_rmse_gaussian_m"]
    # the 2 m fallback replaces only tiles whose predicted excess error over the Gaussian
    # fill is large, so it must not make the learned fill worse
    assert after["height_rmse_with_fallback_m"] <= after["height_rmse_learned_m"]


def test_backward_reads_the_forward_input_even_when_the_caller_dropped_it(lsb):
    """The native backward reads the forward's input again (first-layer weight
    gradients).  Through FillerFn / PaperCNNFn a temporary input stays alive until the
    backward: freeing it and reusing its memory (here: filled with NaN) before the
    backward must not change the gradients."""
    import torch
    from paper_2509_20198_b300 import train as T
    f = lsb.Filler(max_batch=4)
    T.init_params(f, seed=11)
    f.params[-5:] = 0.01
    cnn = lsb.PaperCNN(res=128, max_batch=2)
    T.init_cnn_params(cnn, seed=12)
    for net, fn, shape in ((f, lsb.FillerFn, (4, 64, 64, 8)), (cnn, lsb.PaperCNNFn, (2, 128, 128, 8))):
        xk = torch.zeros(shape, dtype=torch.int16, device="cuda")
        xk[..., :5] = torch.rand(shape[:3] + (5,), device="cuda").to(torch.bfloat16).view(torch.int16)
        grads = []
        for keep in (True, False):
            p = net.params.detach().requires_grad_(True)
            y = fn.apply(p, xk if keep else xk.clone(), net)    # the clone is dropped at once
            junk = torch.full(shape, 0x7FC0, dtype=torch.int16, device="cuda")  # the freed block, bf16 NaN
            w = torch.linspace(-1.0, 1.0, y.numel(), device="cuda").view_as(y)
            (y * w).sum().backward()
            del junk
            grads.append(p.grad.clone())
        assert torch.isfinite(grads[0]).all()
        assert torch.equal(grads[0], grads[1])
