"""Host logic of the autotuner table (no GPU)."""
from paper_2609_08800_gb300 import tune


def test_m_bucket():
    assert tune.m_bucket(12) == 32
    assert tune.m_bucket(32) == 32
    assert tune.m_bucket(120) == 128
    assert tune.m_bucket(216) == 224


def test_store_and_reload(tmp_path):
    p = tmp_path / "t.json"
    tune.store("f32:m128:dev", {"threads": 64}, p)
    tune.store("f64:m128:dev", {"threads": 128}, p)
    t = tune._load(p)
    assert t["f32:m128:dev"]["threads"] == 64 and t["f64:m128:dev"]["threads"] == 128
    assert tune._load(tmp_path / "missing.json") == {}
