"""Autotuner host logic (no GPU): candidate sets per kernel, cache keys and
the JSON cache round trip; and the C ABI's validation of launch tuning."""
import os

import numpy as np
import pytest

from paper_2010_08482_gb300 import autotune, ctq
from paper_2010_08482_gb300 import workloads as w


@pytest.fixture(scope="module")
def imps():
    return {"t2g": ctq.build_impurity(w.model_t2g(), device=-1),
            "hubbard2": ctq.build_impurity(w.model_hubbard2(), device=-1)}


def test_engine_selection(imps):
    assert autotune.engine(imps["t2g"], ctq.FP64) == "fp64"
    assert autotune.engine(imps["t2g"], ctq.TF32X3) == "tc"
    assert autotune.engine(imps["t2g"], ctq.BF16X3) == "tc"


def test_candidates_start_with_default_and_are_unique(imps):
    for prec in (ctq.FP64, ctq.TF32, ctq.TF32X3, ctq.BF16X3):
        c = autotune.candidates(imps["t2g"], prec)
        assert c[0] == {}
        keys = [tuple(sorted(x.items())) for x in c]
        assert len(keys) == len(set(keys))
        for x in c:
            assert set(x) <= set(ctq.TUNE_KEYS)
            if "threads_per_cta" in x:
                assert x["threads_per_cta"] % 32 == 0 and 32 <= x["threads_per_cta"] <= 512
    assert autotune.candidates(imps["t2g"], ctq.TF32X3) == [{}]  # one CTA per SM, nothing to choose
    assert {"ctas_per_sm": 1} in autotune.candidates(imps["t2g"], ctq.BF16X3)


def test_cache_key_buckets_batch_shape(imps):
    k1 = autotune.cache_key(imps["t2g"], ctq.FP64, 4096, 140, 8, False, "GPU")
    k2 = autotune.cache_key(imps["t2g"], ctq.FP64, 4000, 130, 8, False, "GPU")
    k3 = autotune.cache_key(imps["t2g"], ctq.FP64, 8192, 140, 8, False, "GPU")
    k4 = autotune.cache_key(imps["hubbard2"], ctq.FP64, 4096, 140, 8, False, "GPU")
    k5 = autotune.cache_key(imps["t2g"], ctq.TF32X3, 4096, 140, 8, False, "GPU")
    assert k1 == k2 and k1 != k3 and k1 != k4 and k1 != k5


def test_cache_round_trip(tmp_path):
    path = os.path.join(tmp_path, "sub", "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache(path, {"k": {"best": {"threads_per_cta": 64}, "ms": 1.0}})
    assert autotune.load_cache(path)["k"]["best"] == {"threads_per_cta": 64}
    with open(path, "w") as f:
        f.write("not json")
    assert autotune.load_cache(path) == {}


def test_tuning_keys_marshalled():
    o = ctq._opts(ctq.FP64, tune={"threads_per_cta": 64, "ctas_per_sm": 4, "stages": 3, "tile_order": 2})
    assert (o.threads_per_cta, o.ctas_per_sm, o.stages, o.tile_order) == (64, 4, 3, 2)
    with pytest.raises(ValueError):
        ctq._opts(ctq.FP64, tune={"warps": 2})


@pytest.mark.parametrize("bad", [{"threads_per_cta": 48}, {"threads_per_cta": 544}, {"stages": 1},
                                 {"tile_order": 4}, {"ctas_per_sm": -1}])
def test_out_of_range_tuning_rejected_before_any_launch(imps, bad):
    """The tuning fields are validated on the host before anything else of
    the call (a host-only impurity would otherwise fail for lack of a device
    copy), so the message names them."""
    imp = imps["t2g"]
    with pytest.raises(ctq.CtqError, match="launch tuning"):
        ctq.eval_traces(imp, 1, 1.0, 1, 1, 1, None, 1, 1, 1, None, 256, 1 << 20, 0, tune=bad)
    with pytest.raises(ctq.CtqError, match="no device copy"):  # a valid tuning passes validation
        ctq.eval_traces(imp, 1, 1.0, 1, 1, 1, None, 1, 1, 1, None, 256, 1 << 20, 0, tune={"stages": 2})
