"""The serving runtime: handle cache with admission cap (CPU, fake handles) and a small
request trace through the library (GPU)."""
import threading
import time

import numpy as np
import pytest

from paper_2303_08881_gb300 import problems as P
from paper_2303_08881_gb300 import serve as S


class FakeHandle:
    def __init__(self, name):
        self.name = name
        self.freed = False


def _cache(cap):
    freed = []
    c = S.HandleCache(cap, free_fn=lambda h: (setattr(h, "freed", True), freed.append(h.name)))
    return c, freed


def _build(c, key, nbytes):
    assert c.acquire(key) is None
    c.reserve(nbytes)
    h = FakeHandle(key)
    c.insert(key, h, nbytes, nbytes)
    return h


def test_admission_evicts_least_recently_used_idle_handles():
    c, freed = _cache(100)
    for k in "abc":
        _build(c, k, 30)
        c.release(k)
    assert c.held() == 90
    h = c.acquire("a")  # a becomes most recently used
    c.release("a")
    assert h.name == "a" and c.hits == 1
    _build(c, "d", 30)  # needs 20 more bytes: b (least recently used) goes
    assert freed == ["b"] and c.held() == 90 and c.evictions == 1
    c.release("d")
    _build(c, "e", 60)  # c then a
    assert freed == ["b", "c", "a"]
    assert c.peak <= 100


def test_busy_handles_are_not_evicted_and_requests_wait_for_memory():
    c, freed = _cache(100)
    _build(c, "a", 70)  # stays busy
    done = []

    def second():
        _build(c, "b", 50)
        done.append(time.perf_counter())

    t = threading.Thread(target=second)
    t0 = time.perf_counter()
    t.start()
    time.sleep(0.2)
    assert not done and freed == []  # a is busy: b waits
    c.release("a")
    t.join(5)
    assert done and done[0] - t0 >= 0.2 and freed == ["a"]


def test_a_handle_serves_one_request_at_a_time_and_is_built_once():
    c, _ = _cache(1000)
    assert c.acquire("m") is None  # this request builds m
    got = []

    def other():
        got.append(c.acquire("m"))  # waits for the build, then for the handle

    t = threading.Thread(target=other)
    t.start()
    time.sleep(0.1)
    assert not got
    c.reserve(10)
    h = FakeHandle("m")
    c.insert("m", h, 10, 10)
    time.sleep(0.1)
    assert not got  # built but still busy with the builder
    c.release("m")
    t.join(5)
    assert got == [h] and c.hits == 1


def test_oversized_request_is_refused():
    c, _ = _cache(100)
    with pytest.raises(MemoryError):
        c.reserve(101)


def test_failed_build_lets_the_next_request_build():
    c, _ = _cache(100)
    assert c.acquire("k") is None
    c.abandon("k")
    assert c.acquire("k") is None


def test_serving_trace_mix():
    tr = P.serving_trace(400, seed=3)
    kinds = [r.kind for r in tr]
    assert 0.4 < kinds.count("2d") / len(tr) < 0.6
    keys = [r.key for r in tr]
    repeats = len(keys) - len(set(keys))
    assert 0.2 < repeats / len(tr) < 0.4
    arr = np.array([r.arrival for r in tr])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.r_[0.0, arr])
    assert abs(gaps.mean() - 1 / 200) < 1e-3
    for r in tr:
        assert (32 <= r.side <= 512) if r.kind == "2d" else (16 <= r.side <= 96)
        assert 1e-4 <= r.eps <= 1.0


def test_estimate_covers_the_fgmres_basis():
    n, nnz = 100_000, 900_000
    assert S.estimate_bytes(n, nnz, 50) > (2 * 50 + 1) * 8 * n


@pytest.mark.gpu
def test_small_trace_through_the_library():
    import __graft_entry__ as g
    g.build()
    specs = [P.RequestSpec(0, 0.00, "a", "2d", 48, 1e-2, 0.3, 1, 1),
             P.RequestSpec(1, 0.01, "b", "3d", 16, 1e-1, 0.0, 1, 2),
             P.RequestSpec(2, 0.02, "a", "2d", 48, 1e-2, 0.3, 1, 3),
             P.RequestSpec(3, 0.03, "c", "2d", 96, 1e-3, 1.0, 2, 4),
             P.RequestSpec(4, 0.04, "b", "3d", 16, 1e-1, 0.0, 1, 5),
             P.RequestSpec(5, 0.05, "a", "2d", 48, 1e-2, 0.3, 1, 6)]
    reqs = [S.Request(s.rid, s.arrival, s.key, P.problem_of_request(s)) for s in specs]
    rep = S.serve(reqs, workers=3, cap_bytes=8 << 30)
    st = rep.stats
    assert st["completed"] == 6 and st["converged"] == 6, st
    assert st["max_rel_res"] <= 1e-8
    assert st["reused"] >= 1 and rep.cache_hits == st["reused"]
    assert all(r.done >= r.arrival for r in rep.records)
    # a cap just above the largest request's estimate: building it must evict the
    # cached smaller handles (each holds at least its ~2 MB FGMRES basis), and every
    # request still completes
    cap = S.estimate_bytes(96 * 96, 9 * 96 * 96, 50) + (2 << 20)
    rep2 = S.serve(reqs, workers=2, cap_bytes=cap)
    assert rep2.stats["completed"] == 6 and rep2.stats["converged"] == 6
    assert rep2.evictions >= 1 and rep2.peak_bytes <= cap


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix():
    """Requests served concurrently (shared handles, overlapping streams, cache reuse) give
    bit-identical solutions to the same requests solved one at a time on fresh handles:
    every device reduction has a fixed order and each handle owns its stream and graph."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as ilu
    specs = [P.RequestSpec(0, 0.00, "a", "2d", 64, 1e-2, 0.3, 1, 1),
             P.RequestSpec(1, 0.00, "b", "3d", 20, 1e-1, 0.0, 1, 2),
             P.RequestSpec(2, 0.00, "a", "2d", 64, 1e-2, 0.3, 1, 3),
             P.RequestSpec(3, 0.00, "c", "2d", 96, 1e-3, 1.0, 2, 4),
             P.RequestSpec(4, 0.00, "b", "3d", 20, 1e-1, 0.0, 1, 5),
             P.RequestSpec(5, 0.00, "c", "2d", 96, 1e-3, 1.0, 2, 6)]
    reqs = [S.Request(s.rid, s.arrival, s.key, P.problem_of_request(s)) for s in specs]
    mixed = S.serve(reqs, workers=4, cap_bytes=8 << 30, keep_solutions=True)
    assert mixed.stats["completed"] == 6 and mixed.stats["reused"] >= 1
    for rec, rq in zip(mixed.records, reqs):
        pr = rq.problem
        h = ilu.ilu_setup_problem(pr, ilu.Opts())
        b = torch.from_numpy(pr.b).cuda()
        x = torch.zeros_like(b)
        info = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=50, maxit=5000)
        h.close()
        assert info["iters"] == rec.iters
        assert np.array_equal(x.cpu().numpy(), rec.x), rec.rid


@pytest.mark.gpu
def test_unconverged_request_continues_with_a_longer_restart():
    """A solve that reaches maxit continues from its last iterate with a longer restart. On an
    anisotropic request (eps = 1e-3), FGMRES(256) from zero needs n_full steps; with a budget
    of n_full + 10 steps FGMRES(2) does not converge and is reported as not converged, and
    with the escalation to FGMRES(256) (a fresh budget, from the FGMRES(2) iterate) it does."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as ilu
    spec = P.RequestSpec(0, 0.0, "c", "2d", 96, 1e-3, 1.0, 2, 4)
    pr = P.problem_of_request(spec)
    h = ilu.ilu_setup_problem(pr, ilu.Opts())
    b = torch.from_numpy(pr.b).cuda()
    x = torch.zeros_like(b)
    full = ilu.gmres_solve(h, b, x, rtol=1e-8, restart=256, maxit=2000)
    h.close()
    assert full["status"] == 0
    budget = full["iters"] + 10
    reqs = [S.Request(spec.rid, spec.arrival, spec.key, pr)]
    plain = S.serve(reqs, workers=1, restart=2, maxit=budget, escalate=())
    assert plain.records[0].status == 5 and plain.records[0].escalations == 0
    esc = S.serve(reqs, workers=1, restart=2, maxit=budget, escalate=(256,))
    r = esc.records[0]
    assert r.escalations == 1 and r.status == 0 and r.rel_res <= 1e-8, (r.status, r.rel_res, r.iters)
    assert r.iters > budget
