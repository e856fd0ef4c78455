"""The autotuner's host logic (no GPU): candidate sets and the cache key's size classes."""
import pytest

pytest.importorskip("numpy")
from paper_2604_14650_gb300.autotune import candidates, size_class  # noqa: E402


def test_candidates_cover_formats_depths_and_launch_shapes():
    c = candidates(depth=6, auto_levels=4)
    assert {x["format"] for x in c} == {"f8x128", "f8v7", "f16hi"}
    assert {(x["format"], x["kernel"]) for x in c} >= {("f16hi", "hybrid"), ("f16hi", "coop")}
    assert {x["smem_levels"] for x in c if x["kernel"] == "hybrid" and x["format"] != "f16hi"} == {3, 4}
    assert {(x["block_threads"], x["ctas_per_sm"]) for x in c
            if x["kernel"] == "hybrid" and x["format"] != "f16hi"} == {(512, 0), (256, 0), (512, 1)}


def test_persistent_candidates_stay_in_the_single_launch():
    c = candidates(depth=6, auto_levels=4, persistent=True)
    assert c and all(x["kernel"] == "hybrid" for x in c)
    assert {x["format"] for x in c} == {"f8x128", "f8v7", "f16hi"}
    assert all("block_threads" not in x for x in c)
    assert candidates(depth=3, auto_levels=0, persistent=True) == [
        dict(format="f8x128", kernel="hybrid", smem_levels=0),
        dict(format="f8v7", kernel="hybrid", smem_levels=0),
        dict(format="f16hi", kernel="hybrid", smem_levels=-1)]
    # with the F16HI layout's automatic depth known, that depth and one shallower
    c16 = [x for x in candidates(depth=6, auto_levels=4, persistent=True, auto16=4)
           if x["format"] == "f16hi"]
    assert [x["smem_levels"] for x in c16] == [3, 4]


def test_size_classes_are_half_octaves():
    assert size_class(1024) == 10.0
    assert size_class(1448) == 10.5          # 2^10.5 = 1448.2
    assert size_class(2048) == 11.0
    assert size_class(0) == size_class(2) == 1.0


def test_benchmark_reads_recorded_counters_safely():
    """bench.py's reader of profiles/traffic.json answers a dict or None for every kernel listed
    there (and for an unknown one), never raises."""
    import json
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    path = os.path.join(root, "profiles", "traffic.json")
    names = list(json.load(open(path))) if os.path.exists(path) else []
    for name in names + ["no such kernel"]:
        r = bench.recorded_counters(name)
        assert r is None or isinstance(r, dict)
