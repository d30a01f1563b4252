"""Autotuner selection and cache logic (no GPU: a fake timer stands in for CUDA events)."""
from paper_2408_02758_gb300 import autotune as A


def test_pick_returns_fastest_and_skips_failures():
    times = {64: 3.0, 128: 1.5, 256: 2.0}

    def timer(c):
        if c["b"] == 512:
            raise RuntimeError("launch failed")
        return times[c["b"]]

    ch = A.pick([{"b": 64}, {"b": 512}, {"b": 128}, {"b": 256}], timer)
    assert ch.params == {"b": 128} and ch.ms == 1.5


def test_cache_round_trip(tmp_path):
    p = tmp_path / "tune.json"
    c = A.Cache(p)
    key = A.shape_key("GB300", "compute", 2, 0, "fp32c", 2_097_152, 1500)
    assert c.get(key) is None
    c.put(key, A.Choice({"advect_block": 128}, 1.25))
    c2 = A.Cache(p)
    got = c2.get(key)
    assert got.params == {"advect_block": 128} and got.ms == 1.25


def test_shape_key_buckets():
    k1 = A.shape_key("G", "compute", 2, 0, "fp32c", 2_000_000, 1500)
    k2 = A.shape_key("G", "compute", 2, 0, "fp32c", 1_500_000, 1024)
    k3 = A.shape_key("G", "compute", 2, 0, "fp32c", 4_200_000, 1500)
    assert k1 == k2 and k1 != k3
