"""Serving with continuous batching (idet_server_*): every result equals the
determinant computed alone (and the oracle's where it is affordable), jobs
overlap and are batched, admission respects the device-memory budget."""
import numpy as np
import pytest

import workloads
from oracle import exact

pytestmark = pytest.mark.gpu

idet = pytest.importorskip("paper_cs_0511066_b300")


def _job(g, nmax):
    return workloads.serving_job(g, nmin=16, nmax=nmax)


def test_server_results_same_alone_and_in_the_mix():
    g = workloads.rng(21)
    mats = [_job(g, 700) for _ in range(40)]
    mats += [workloads.dense_pm100(30, seed=3), np.zeros((9, 9), dtype=np.int64)]
    with idet.Server(slots=3, max_batch=16) as srv:
        tickets = [srv.submit(A) for A in mats]
        res = [srv.poll(t) for t in tickets]
        st = srv.info()
    assert st["completed"] == len(mats)
    for A, (d, info) in zip(mats, res):
        assert d == idet.int_det(A), A.shape
        if A.shape[0] <= 40:
            assert d == exact.bareiss_det(A.tolist())
        assert info["status"] == 0 and info["ms_latency"] >= info["ms_run"] >= 0
    assert any(info["batched"] > 1 for _, info in res)
    assert st["max_running"] >= 2
    # some work of different workers overlapped in time
    spans = sorted((i["t_start_ms"], i["t_end_ms"], i["worker"]) for _, i in res)
    assert any(a[2] != b[2] and b[0] < a[1] for a, b in zip(spans, spans[1:]))


def test_server_admission_by_memory_budget():
    """A budget that holds one n = 1024 job (and small ones) at a time: the
    two large jobs never run together, small jobs are admitted beside them."""
    g = workloads.rng(5)
    big = [g.integers(-1000, 1000, size=(1024, 1024), endpoint=True, dtype=np.int64)
           for _ in range(2)]
    small = [g.integers(-1000, 1000, size=(64, 64), endpoint=True, dtype=np.int64)
             for _ in range(6)]
    one_big = int(1024 * 1024 * 120 + (16 << 20))
    budget = one_big + 4 * int(64 * 64 * 120 + (16 << 20))
    with idet.Server(hbm_budget=budget, slots=3, small_n=128, max_batch=2) as srv:
        tb = [srv.submit(A) for A in big]
        ts = [srv.submit(A) for A in small]
        rb = [srv.poll(t) for t in tb]
        rs = [srv.poll(t) for t in ts]
    (d0, i0), (d1, i1) = rb
    assert d0 == idet.int_det(big[0]) and d1 == idet.int_det(big[1])
    assert i0["t_end_ms"] <= i1["t_start_ms"] or i1["t_end_ms"] <= i0["t_start_ms"]
    for A, (d, _) in zip(small, rs):
        assert d == idet.int_det(A)


def test_server_timeout_and_oversized_job():
    g = workloads.rng(9)
    A = g.integers(-(1 << 20), 1 << 20, size=(1500, 1500), endpoint=True, dtype=np.int64)
    B = workloads.dense_pm100(50, seed=1)
    with idet.Server(slots=1, small_n=0) as srv:
        ta = srv.submit(A)
        tb = srv.submit(B)          # queued behind A on the only worker
        assert srv.poll(tb, timeout_ms=0) is None
        assert srv.poll(ta)[0] == idet.int_det(A)
        assert srv.poll(tb)[0] == exact.bareiss_det(B.tolist())
    with idet.Server(hbm_budget=1 << 26, slots=1) as srv:
        with pytest.raises(idet.IdetError):
            srv.submit(np.ones((2000, 2000), dtype=np.int64))


def test_server_same_ticket_polled_from_two_threads():
    """Two threads wait on one ticket: one collects the determinant, the
    other returns an error instead of reading a collected job."""
    import threading
    A = workloads.dense_pm100(300, seed=4)
    want = idet.int_det(A)
    out = []
    with idet.Server(slots=1) as srv:
        t = srv.submit(A)

        def waiter():
            try:
                out.append(("ok", srv.poll(t)[0]))
            except idet.IdetError as e:
                out.append(("err", e.code))

        th = [threading.Thread(target=waiter) for _ in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join(timeout=60)
        assert not any(x.is_alive() for x in th)
    assert sorted(o[0] for o in out) == ["err", "ok"]
    assert [o[1] for o in out if o[0] == "ok"] == [want]
    assert [o[1] for o in out if o[0] == "err"] == [1]
