"""Host logic of the launch-schedule autotuner (no device): shape keys and the cache."""
import numpy as np

from paper_2202_02264_gb300 import autotune as A, workloads as W


def test_shape_key_depends_on_the_shape_not_the_order():
    m = W.lgssm_d4()
    k1 = A.shape_key(m, [64, 100, 4096], 512, 2, "dev")
    assert k1 == A.shape_key(m, [4096, 64, 100], 512, 2, "dev")
    assert k1 != A.shape_key(m, [64, 100, 4095], 512, 2, "dev")
    assert k1 != A.shape_key(m, [64, 100, 4096], 1024, 2, "dev")
    assert k1 != A.shape_key(m, [64, 100, 4096], 512, 0, "dev")
    assert k1 != A.shape_key(W.lgssm_d8(), [64, 100, 4096], 512, 2, "dev")


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setattr(A, "_CACHE", str(tmp_path / "a" / "autotune.json"))
    assert A._load_cache() == {}
    A._store_cache({"k": {"fused_max_merges": 32, "max_merges_per_launch": 4096}})
    assert A._load_cache()["k"]["max_merges_per_launch"] == 4096


def test_candidates_cover_never_fused_and_the_default():
    assert -1 in A.FUSED_CANDIDATES and 32 in A.FUSED_CANDIDATES
    assert 1024 in A.CHUNK_CANDIDATES
