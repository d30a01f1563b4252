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


def test_gradient_choice_cached_per_layout(tmp_path, monkeypatch):
    """params_for_gradient keys its cache by the mesh's neighbour layout: a stored choice for CSR
    rows comes back without timing anything, and a fixed-width-list mesh of the same size misses
    it (and would be timed)."""
    monkeypatch.setattr(A, "_gpu_name", lambda: "GB300")

    class Desc:
        def __init__(self, ell_width, stencil=0):
            self.ell_width, self.stencil = ell_width, stencil

    class Mesh:
        def __init__(self, ell_width):
            self.desc, self.dim, self.n_nodes = Desc(ell_width), 3, 16_777_216

    cache = A.Cache(tmp_path / "tune.json")
    key = A.shape_key("GB300", "gradient-csr", 3, 0, "fp32c", 16_777_216, 1)
    cache.put(key, A.Choice({"grad_staging": 0}, 0.66))

    def no_timing(*a, **k):
        raise AssertionError("timed although cached")

    monkeypatch.setattr(A, "_pick_gradient", no_timing)
    assert A.params_for_gradient(Mesh(0), None, "fp32c", 5.0, cache=cache) == {"grad_staging": 0}
    timed = []
    monkeypatch.setattr(A, "_pick_gradient", lambda *a, **k: timed.append(1) or A.Choice({"grad_staging": 1}, 0.55))
    assert A.params_for_gradient(Mesh(14), None, "fp32c", 5.0, cache=cache) == {"grad_staging": 1}
    assert timed == [1]
    assert A.Cache(tmp_path / "tune.json").get(A.shape_key("GB300", "gradient-ell", 3, 0, "fp32c", 16_777_216, 1))
