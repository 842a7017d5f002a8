"""Host logic of the serving loop (no device): first-come-first-served admission under a
byte budget without overtaking, a lane's tick capacity, stage progression through
Algorithm 2, every level of Algorithm 6 and the resolve, and memory released only when a
request's results are out."""
import numpy as np
import pytest

from paper_2202_02264_gb300 import serving as S, workloads as W


def _req(rid, K, lane="a", arrival=0.0, N=8):
    return S.Request(rid, lane, W.lgssm_1d(), N, np.zeros((K, 1)), 1, arrival)


def test_levels_and_merges_follow_the_schedule():
    # left-aligned 2^l blocks; a block without a right partner passes through (Algorithm 6)
    assert [S.levels(K) for K in (1, 2, 3, 4, 5, 1024, 1025)] == [0, 1, 2, 2, 3, 10, 11]
    for K in (1, 2, 3, 7, 64, 100, 1025):
        assert sum(S.merges_at_level(K, l) for l in range(S.levels(K))) == K - 1
    assert [S.merges_at_level(5, l) for l in range(3)] == [2, 1, 1]


def test_admission_is_fifo_under_the_budget():
    sch = S.Scheduler(100, lambda r: r.K)
    for rid, K in enumerate([40, 50, 30, 5]):
        sch.submit(_req(rid, K))
    got = [s.req.rid for s in sch.admit(0.0)]
    assert got == [0, 1]                 # 40 + 50 fit; 30 waits, and 5 may not overtake it
    assert sch.used == 90 and len(sch.queue) == 2
    assert sch.admit(0.0) == []


def test_arrivals_in_the_future_wait():
    sch = S.Scheduler(10**9, lambda r: r.K)
    sch.submit(_req(0, 4, arrival=0.0))
    sch.submit(_req(1, 4, arrival=5.0))
    assert [s.req.rid for s in sch.admit(1.0)] == [0]
    assert [s.req.rid for s in sch.admit(5.0)] == [1]


def test_stages_run_init_levels_resolve_then_release():
    sch = S.Scheduler(1000, lambda r: 100)
    sch.submit(_req(0, 5))               # L = 3: stages -1, 0, 1, 2, 3
    sch.submit(_req(1, 1))               # L = 0: stages -1, 0
    sch.admit(0.0)
    seen = {0: [], 1: []}
    done = []
    for _ in range(10):
        for s in sch.tick_plan("a"):
            seen[s.req.rid].append(s.stage)
        done += sch.advance("a")
    assert seen[0] == [-1, 0, 1, 2, 3] and seen[1] == [-1, 0]
    assert sorted(s.req.rid for s in done) == [0, 1]
    assert sch.used == 200 and sch.busy()          # results not out yet: memory still held
    for s in done:
        sch.release(s)
    assert sch.used == 0 and not sch.busy()


def test_freed_memory_admits_the_next_request():
    sch = S.Scheduler(100, lambda r: 60)
    sch.submit(_req(0, 3))
    sch.submit(_req(1, 3))
    assert [s.req.rid for s in sch.admit(0.0)] == [0]
    finished = []
    while not finished:
        sch.tick_plan("a")
        finished = sch.advance("a")
    assert sch.admit(0.0) == []          # still held until released
    sch.release(finished[0])
    assert [s.req.rid for s in sch.admit(0.0)] == [1]


def test_lane_tick_capacity():
    sch = S.Scheduler(10**9, lambda r: 1, lane_limit=lambda lane: 10)
    sch.submit(_req(0, 16))              # 8 combinations at level 0
    sch.submit(_req(1, 8))               # 4 more would exceed 10
    sch.submit(_req(2, 4, lane="b"))     # another lane has its own capacity
    assert [s.req.rid for s in sch.admit(0.0)] == [0]
    with pytest.raises(ValueError):
        sch.submit(_req(3, 64))          # can never fit one tick


def test_request_bytes_counts_every_buffer():
    K, N, d = 100, 64, 8
    b = S.request_bytes(K, N, d)
    assert b >= K * N * d * 4 + K * N * 4 + (K - 1) * 2 * N * 4 + 16 * K * N
    assert S.request_bytes(K, N, d, gauss_prop=True, conditional=True) > b


def test_request_stream_shape():
    reqs = S.request_stream(200, rate=2000.0, K_range=(64, 512), Ns=(64, 128))
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert 0.05 < arr[-1] < 0.2                      # ~200 / 2000 s
    frac_sv = np.mean([r.lane.startswith("sv") for r in reqs])
    assert 0.15 < frac_sv < 0.45
    assert all(64 <= r.K <= 512 for r in reqs)
