"""Host logic of the serving scheduler (admission by device-memory footprint,
FIFO order, resident-plan cache and eviction) with the fake backend: no GPU."""
import time

import numpy as np
import pytest

from paper_2506_04710_gb300 import build, ztoep


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def dummy():
    return np.zeros(4, np.complex128)


def fp_of(nx, b, e, nrhs):
    """Bytes a host-input request reserves: the footprint plus the device
    staging copies of T, B and C for its plan build."""
    d, _ = ztoep.make_desc(nx, nx, b, e)
    staging = 16 * ((2 * nx - 1) ** 2 * b * b + e * nx * nx * b + e * e)
    return ztoep.ztoep_footprint(d, nrhs, 30) + staging


def submit(s, nx, b, e, nrhs, key=0):
    a = dummy()
    return s.submit((nx, nx, b, e), a, a, a, np.zeros((nrhs, 4), np.complex128), np.zeros((nrhs, 4), np.complex128),
                    plan_key=key, on_device=False)


def test_admission_never_exceeds_budget():
    fp = fp_of(16, 32, 256, 8)
    s = ztoep.Scheduler(hbm_budget=int(2.5 * fp), workers=4, fake_us=20000)
    ids = [submit(s, 16, 32, 256, 8) for _ in range(8)]
    for i in ids:
        rc, st, _ = s.wait(i, 10000)
        assert rc == 0 and st.state == 2 and st.status == 0
    stats = s.stats()
    assert stats.completed == 8 and stats.max_in_flight == 2
    assert stats.peak_bytes <= int(2.5 * fp)
    s.close()


def test_fifo_order_with_one_worker():
    s = ztoep.Scheduler(hbm_budget=1 << 40, workers=1, fake_us=5000)
    ids = [submit(s, 8 + k, 32, 64, 1) for k in range(6)]
    states = [s.wait(i, 10000)[1] for i in ids]
    q = [st.queue_ms for st in states]
    assert q == sorted(q)
    assert all(st.latency_ms >= st.queue_ms for st in states)
    s.close()


def test_concurrency_up_to_workers():
    s = ztoep.Scheduler(hbm_budget=1 << 40, workers=3, fake_us=30000)
    ids = [submit(s, 8, 32, 64, 1) for _ in range(9)]
    for i in ids:
        s.wait(i, 10000)
    assert s.stats().max_in_flight == 3
    s.close()


def test_rejects_oversized_and_bad_requests():
    fp = fp_of(32, 64, 512, 4)
    s = ztoep.Scheduler(hbm_budget=fp // 2, workers=2, fake_us=1000)
    with pytest.raises(ztoep.ZtoepError) as e:
        submit(s, 32, 64, 512, 4)
    assert e.value.status == ztoep.ZTOEP_ERR_NOMEM
    with pytest.raises(ztoep.ZtoepError) as e:
        submit(s, 0, 64, 16, 1)
    assert e.value.status == ztoep.ZTOEP_ERR_ARG
    s.close()


def test_resident_plans_are_reused_and_evicted_lru():
    fp = fp_of(16, 32, 256, 4)
    # room for one running request plus about one idle resident plan
    s = ztoep.Scheduler(hbm_budget=int(1.6 * fp), workers=1, fake_us=2000)
    order = [1, 1, 2, 1, 3, 3]
    states = []
    for key in order:
        rid = submit(s, 16, 32, 256, 4, key=key)
        states.append(s.wait(rid, 10000)[1])
    st = s.stats()
    # key 1 survives the admission of key 2 (plan 2 is the LRU victim when key 1
    # returns), plan 1 is evicted when key 3 comes back
    assert [x.plan_reused for x in states] == [0, 1, 0, 1, 0, 1]
    assert st.plans_built == 3 and st.plans_reused == 3 and st.plans_evicted == 2
    assert st.peak_bytes <= int(1.6 * fp)
    s.close()


def test_inputs_released_once_consumed():
    s = ztoep.Scheduler(hbm_budget=1 << 40, workers=1, fake_us=30000)
    a = submit(s, 8, 32, 64, 1)
    b = submit(s, 8, 32, 64, 1)
    assert not s.drop_inputs(b)  # still queued behind a: its blocks are needed
    s.wait(b, 10000)
    assert s.drop_inputs(a) and s.drop_inputs(b)
    assert s._keep[b][1] is None and s._keep[b][4] is not None  # V, X kept
    assert s.poll(b).inputs_consumed == 1
    s.close()


def test_grouping_takes_consecutive_compatible_requests():
    """group_max = 4 with one worker: the head and the three compatible
    requests behind it run as one group; a request with a key already in the
    group (its plan would be shared) ends the group, FIFO order is kept."""
    s = ztoep.Scheduler(hbm_budget=1 << 40, workers=1, fake_us=20000, group_max=4)
    t0 = time.perf_counter()
    subs = [(submit(s, 8, 32, 64, 1), time.perf_counter())]  # runs alone: taken before the rest is queued
    for k in (11, 12, 13, 14, 14, 15):
        subs.append((submit(s, 8, 32, 64, 2, key=k), time.perf_counter()))
    states = [s.wait(i, 10000)[1] for i, _ in subs]
    assert all(st.state == 2 and st.status == 0 for st in states)
    st = s.stats()
    assert st.completed == 7 and st.groups >= 1
    # FIFO: start times (submission + time queued) never go back in arrival order
    starts = [1e3 * (t - t0) + x.queue_ms for (_, t), x in zip(subs, states)]
    assert all(b >= a - 1.0 for a, b in zip(starts, starts[1:]))
    s.close()


def test_grouping_respects_size_ratio_and_budget():
    fp = fp_of(16, 32, 256, 8)
    s = ztoep.Scheduler(hbm_budget=int(2.5 * fp), workers=1, fake_us=10000, group_max=8)
    ids = [submit(s, 16, 32, 256, 8) for _ in range(6)]
    for i in ids:
        assert s.wait(i, 10000)[0] == 0
    st = s.stats()
    assert st.max_in_flight <= 2 and st.peak_bytes <= int(2.5 * fp)
    s.close()
    # a request over 4x the head's size does not join its group
    s = ztoep.Scheduler(hbm_budget=1 << 40, workers=1, fake_us=10000, group_max=8)
    a = submit(s, 8, 32, 64, 1)
    b = submit(s, 8, 32, 64, 1)
    c = submit(s, 8, 32, 64, 64)
    for i in (a, b, c):
        assert s.wait(i, 10000)[0] == 0
    assert s.stats().max_in_flight <= 2
    s.close()
