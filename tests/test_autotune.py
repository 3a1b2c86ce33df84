"""Autotuner host logic (no GPU): the candidate leaf sizes bracket the paper's tabulated
optimum (Table 10), keys separate workloads by size class, and the JSON cache round-trips."""
import os

from paper_2508_02626_gb300 import autotune as A


def test_paper_table_and_candidates():
    assert [A.paper_leaf_size(p) for p in (2, 4, 6, 8, 10)] == [64, 128, 256, 256, 512]
    assert A.paper_leaf_size(5) == 256 and A.paper_leaf_size(0) == 64 and A.paper_leaf_size(9) == 512
    for p in range(11):
        c = A.leaf_candidates(p)
        assert c == sorted(set(c)) and c[-1] == A.paper_leaf_size(p) and min(c) >= 8
        assert len(c) >= 4


def test_size_class_and_key():
    assert A.size_class(1 << 20, 1) == A.size_class((1 << 20) + 5, 1)
    assert A.size_class(1 << 20, 1) != A.size_class(1 << 22, 1)
    assert A.size_class(1 << 22, 256) != A.size_class(1 << 22, 1)
    assert A.make_key("GB300", 6, "fp32", 1000, 2) != A.make_key("GB300", 8, "fp32", 1000, 2)


def test_cache_round_trip(tmp_path):
    path = os.path.join(str(tmp_path), "sub", "tune.json")
    c = A.Cache(path)
    assert c.get("k") is None
    c.put("k", {"max_leaf": 32, "leaf_warps": 4, "ms": 1.5})
    c2 = A.Cache(path)
    assert c2.get("k") == {"max_leaf": 32, "leaf_warps": 4, "ms": 1.5}
    with open(path, "w") as f:
        f.write("{not json")
    assert A.Cache(path).get("k") is None  # a damaged cache is ignored, not fatal
