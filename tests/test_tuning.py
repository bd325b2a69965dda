"""The autotuner's launch-shape cache (host logic only)."""
import json

import paper_0904_0642_gb300 as su3
from paper_0904_0642_gb300 import tuning


def cfg(**kw):
    base = dict(dims=[8, 8, 8, 8], storage=su3.SU3_FP32_12)
    base.update(kw)
    dims = base.pop("dims")
    return su3.make_config(dims, **base)


def test_key_separates_what_the_timings_depend_on():
    v = "libsu3gb300 test sm_103a"
    k = tuning.key_of([cfg()], v)
    assert k == tuning.key_of([cfg(beta=5.5, seed=9, hits=3)], v)  # physics parameters do not matter
    others = [cfg(storage=su3.SU3_FP32_18), cfg(dims=[8, 8, 8, 4]), cfg(dims=[8, 8, 8]),
              cfg(boundary=su3.SU3_DLT), cfg(boundary=su3.SU3_DLT, glue_mask=0b1000),
              cfg(ndiv=[2, 1, 1, 1]), cfg(boundary=su3.SU3_DLT, beta1=4.0)]
    keys = {tuning.key_of([c], v) for c in others}
    assert k not in keys and len(keys) == len(others)
    assert tuning.key_of([cfg()], "another build") != k
    # ensembles: the chain count and every distinct shape
    assert tuning.key_of([cfg()] * 3, v) != tuning.key_of([cfg()] * 4, v)
    mixed = tuning.key_of([cfg(), cfg(dims=[4, 4, 4, 4])], v)
    assert "4x4x4x4" in mixed and "8x8x8x8" in mixed


def test_store_and_lookup(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tuning.lookup(path, "a") is None
    tuning.store(path, "a", (3, 256, 2, 612.5))
    tuning.store(path, "b", (0, 128, 4, 700.0))
    assert tuning.lookup(path, "a") == (3, 256, 2, 612.5)
    assert tuning.lookup(path, "b") == (0, 128, 4, 700.0)
    tuning.store(path, "a", (0, 64, 0, 600.0))
    assert tuning.lookup(path, "a") == (0, 64, 0, 600.0)
    assert set(json.load(open(path))) == {"a", "b"}


def test_corrupt_cache_is_a_miss_and_is_replaced(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tuning.lookup(str(path), "a") is None
    tuning.store(str(path), "a", (1, 128, 5, 1.0))
    assert tuning.lookup(str(path), "a") == (1, 128, 5, 1.0)
