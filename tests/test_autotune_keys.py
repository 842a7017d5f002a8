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


def test_candidates_search_the_tile_width_and_keep_the_fused_kernel_at_32():
    m = W.lgssm_d4()
    c = A.candidates(m, 512, 2)
    tiles = {t for *_, t in c}
    assert tiles == {32, 64}
    assert all(t == 32 for _, _, tcf, t in c if tcf > 0)        # the fused kernel takes 32
    assert any(tcf > 0 for _, _, tcf, _ in c)                   # eligible: BF16, N <= 512, d <= 4
    assert len(c) == len(set(c))
    # the fused kernel is searched at its own (larger) chunks, the split path at the others
    assert {mc for _, mc, tcf, _ in c if tcf > 0} == set(A.TC_CHUNK_CANDIDATES)
    assert {mc for _, mc, tcf, _ in c if tcf < 0} == set(A.CHUNK_CANDIDATES)
    # FP32 cross term: no fused tensor-core candidates; N = 4096: only the wider tiles
    assert all(tcf < 0 for _, _, tcf, _ in A.candidates(m, 512, 0))
    assert {t for *_, t in A.candidates(m, 4096, 2)} == {64}
