"""Host logic of the launch-shape table (no GPU needed): defaults, keys, pinning,
validation and clearing.  The GPU side (every candidate shape gives the same results,
the autotuners pick one of them) is in test_gpu_tune.py."""
import pytest
import torch


@pytest.fixture(scope="module")
def lsb():
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    build.build_library()
    lsb.tune_clear()
    yield lsb
    lsb.tune_clear()


def _pts(n):
    return {"x": torch.empty(n, dtype=torch.int32)}


def test_defaults(lsb):
    assert lsb.bin_shape(_pts(567_111_960)) == {"spans_per_cta": 16, "prefetch_batches": 2}
    assert lsb.fill_shape(_pts(12_000), n_out=256) == {"split": 4, "ctas_per_sm": 4}
    assert lsb.fill_shape(_pts(1_320_000), n_out=40_000) == {"split": 1, "ctas_per_sm": 4}
    assert lsb.fill_shape(_pts(12_000), n_out=256, res=96) == {"split": 1, "ctas_per_sm": 4}


def test_pinned_shape_applies_to_its_key_only(lsb):
    lsb.set_bin_shape(_pts(1_000_000), shape={"spans_per_cta": 32, "prefetch_batches": 3})
    # same level sizes and floor(log2 n): same key
    assert lsb.bin_shape(_pts(1_048_575)) == {"spans_per_cta": 32, "prefetch_batches": 3}
    # another order of magnitude, other levels: defaults
    assert lsb.bin_shape(_pts(2_100_000)) == {"spans_per_cta": 16, "prefetch_batches": 2}
    assert lsb.bin_shape(_pts(1_000_000), levels=(640,)) == {"spans_per_cta": 16, "prefetch_batches": 2}
    lsb.set_bin_shape(_pts(1_000_000), shape=None)
    assert lsb.bin_shape(_pts(1_000_000)) == {"spans_per_cta": 16, "prefetch_batches": 2}
    lsb.set_fill_shape(_pts(5000), 300, shape={"split": 2, "ctas_per_sm": 1})
    assert lsb.fill_shape(_pts(5000), 300) == {"split": 2, "ctas_per_sm": 1}
    assert lsb.fill_shape(_pts(5000), 300, radius_cm=8000) == {"split": 4, "ctas_per_sm": 4}


@pytest.mark.parametrize("shape", [{"spans_per_cta": 0, "prefetch_batches": 2},
                                   {"spans_per_cta": 257, "prefetch_batches": 2},
                                   {"spans_per_cta": 16, "prefetch_batches": 0},
                                   {"spans_per_cta": 16, "prefetch_batches": 5}])
def test_invalid_bin_shapes_are_rejected(lsb, shape):
    from paper_2509_20198_b300._native import LsError
    with pytest.raises(LsError):
        lsb.set_bin_shape(_pts(10), shape=shape)


@pytest.mark.parametrize("res,shape", [(64, {"split": 3, "ctas_per_sm": 2}),
                                       (64, {"split": 1, "ctas_per_sm": 5}),
                                       (64, {"split": 1, "ctas_per_sm": 0}),
                                       (48, {"split": 4, "ctas_per_sm": 2}),   # 48 is no multiple of 64
                                       (80, {"split": 2, "ctas_per_sm": 2})])  # nor 80 of 32
def test_invalid_fill_shapes_are_rejected(lsb, res, shape):
    from paper_2509_20198_b300._native import LsError
    with pytest.raises(LsError):
        lsb.set_fill_shape(_pts(10), 10, res=res, shape=shape)


def test_clear_forgets_every_entry(lsb):
    lsb.set_bin_shape(_pts(77), shape={"spans_per_cta": 4, "prefetch_batches": 1})
    lsb.set_fill_shape(_pts(77), 7, shape={"split": 1, "ctas_per_sm": 1})
    lsb.tune_clear()
    assert lsb.bin_shape(_pts(77)) == {"spans_per_cta": 16, "prefetch_batches": 2}
    assert lsb.fill_shape(_pts(77), 7) == {"split": 4, "ctas_per_sm": 4}


def test_tuner_rejects_bad_repetitions_before_touching_the_gpu():
    import ctypes
    from paper_2509_20198_b300 import _native as N
    L = N.lib()
    pts = N.LsPoints(None, None, None, None, None, None, 0, None)
    lv = (N.LsBins * 1)(N.LsBins(640, None, None, None, None, None, None, None))
    assert L.ls_tune_bin_points(ctypes.byref(pts), None, lv, 1, None, 0, None, None, None) == -1
    prm = N.LsFillParams(64, 12000, 4000.0)
    assert L.ls_tune_fill_sparse(ctypes.byref(pts), None, ctypes.byref(prm), None, 0, None, None, 1001, None,
                                 None, None) == -1
